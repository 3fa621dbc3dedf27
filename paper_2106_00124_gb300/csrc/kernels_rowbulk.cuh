// kernels_rowbulk.cuh -- the final pass of the row schedule for 4-byte local
// types, staged by the Blackwell bulk-copy engine.
//
// Same result as k_rowx (kernels_rows.cuh): for every row x' = (x_1..x_{d-1})
// of the view [O, n2, L] of its input,
//
//   out[x', x_d] = T[x'] (+) (+)_{y < x_d} H[x', y] (+) (+)_{y >= x_d + k3} H[x', y]
//
// with H the window of width k2 along n2 of the input (Sec. 3, BDBS-Along-Dim
// for dimension d-1; k2 = 1 means no window).  That is the last step of the
// row schedule of box-complement (Sec. 4, the regions of the excluded-sum
// components along dimension d plus the lower-dimensional part T).
//
// Organised for few instructions per element (the pass moves 8 bytes per
// element, so at HBM speed an SM has about 45 issue slots per element, and
// far fewer once latencies are counted):
//   * a persistent grid; a tile is TR consecutive rows of one slice, which
//     are contiguous in memory, so ONE elected thread stages the tile and its
//     k2 - 1 halo rows with a single cp.async.bulk into shared memory
//     (completion on an mbarrier).  NBUF staging buffers: the copies of the
//     next NBUF - 1 tiles are in flight while a tile is computed;
//   * the window along n2 walks 4-element column quads (16-byte shared
//     loads and stores; 2- or 1-element columns for windows over 8) and
//     writes a second, swizzled buffer W, each thread a segment of rows.
//     When k2 is the compile-time width and segments hold whole blocks of
//     k2 rows, the walk has no bounds tests at all;
//   * the row phase gives each of `lpr` lanes a strip of EPL (16 or 32)
//     consecutive elements, so the scans of the strip totals across lanes
//     are short (log2 lpr shuffle steps each way); each lane then writes its
//     inclusive suffixes back into its own strip of W, reads the suffix at
//     x_d + k3 from there, writes its results into the strip, and the warp
//     copies its rows out with coalesced 16-byte stores.
#pragma once

#include <type_traits>

#include "kernels_rows.cuh"

namespace exsum {

// Blocks that gave up a bounded wait on a bulk copy (one counter per
// translation unit; read by exsum_device_timeouts).  Never expected to move.
static __device__ unsigned g_wait_timeouts;

// Every translation unit registers a reader of its own counter with the
// library (exsum_abi.cu), which adds them up.
void register_timeout_reader(unsigned (*reader)());

namespace {
unsigned read_wait_timeouts()
{
    unsigned v = 0;
    if (cudaMemcpyFromSymbol(&v, g_wait_timeouts, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return v;
}
struct WaitTimeoutsReader {
    WaitTimeoutsReader() { register_timeout_reader(&read_wait_timeouts); }
} g_wait_timeouts_reader;
}  // namespace

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}

// Makes the initialised barriers visible to the bulk-copy (async) proxy.
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// Orders this thread's earlier shared-memory accesses (generic proxy) before
// later bulk copies (async proxy) into the same memory.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Global -> shared bulk copy of `bytes` (a multiple of 16, both addresses
// 16-byte aligned); its completion counts `bytes` transactions on `bar`.
__device__ __forceinline__ void bulk_g2s(void *sdst, const void *gsrc, unsigned bytes, uint64_t *bar,
                                         uint64_t pol)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;\n" ::"r"(
            smem_addr(sdst)),
        "l"(__cvta_generic_to_global(gsrc)), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// As mbar_try_wait, letting the hardware suspend the thread for up to
// `ns` nanoseconds while the phase is incomplete (no spinning issue slots).
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, unsigned parity, unsigned ns)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of `bar`: at most 2^16 suspended tries of
// up to 20 us each (about a second), far beyond any copy of a few hundred KB.
// Returns false if the bound ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity)
{
    for (int i = 0; i < (1 << 16); ++i)
        if (mbar_try_wait_sleep(bar, parity, 20000u)) return true;
    return false;
}

// Rows a tile's staging buffer holds.  Block-aligned walk (k2 == KMAX and
// segments of whole blocks): the TR tile rows, the k2 - 1 halo rows and one
// more that the last block's look-ahead reads (its value is not used).
// Otherwise the walk may read up to 2 k2 - 1 rows past a segment start, so
// k2 more rows (identity) follow the halo.
__host__ __device__ inline int rowbulk_stage_rows(int TR, int k2, bool aligned)
{
    return k2 <= 1 ? TR : (aligned ? TR + k2 : TR + 2 * k2 - 1);
}

// Column width of the window walk and the number of row segments per
// column group for a block of nt threads.  Rows whose length is not a
// multiple of 4 (odd) sit at every alignment in the staging buffer: the walk
// reads them one element at a time.
__host__ __device__ constexpr int rowbulk_cw(int kmax, bool odd = false)
{
    return odd ? 1 : (kmax <= 8 ? 4 : (kmax <= 16 ? 2 : 1));
}
__host__ __device__ inline int rowbulk_segs(int L, int kmax, int nt, bool odd = false)
{
    const int lq = L / rowbulk_cw(kmax, odd);
    return lq >= nt ? 1 : nt / lq;
}

// Elements of one staging buffer: the rows, and for odd rows room for the
// shift (0 .. 3 elements) that puts the copy's source on a 16-byte
// boundary, rounded to whole 16-byte chunks.
__host__ __device__ inline int rowbulk_stage_elems(int rows, int L, bool odd)
{
    return odd ? (rows * L + 3 + 3) & ~3 : rows * L;
}

// Shared memory of one block (bytes): NBUF barriers (128 bytes), NBUF
// staging buffers, the row buffer W (TR rows of LSW elements) and a 16-byte
// identity chunk.
__host__ __device__ inline size_t rowbulk_smem(int TR, int k2, bool aligned, int L, int LSW, int nbuf,
                                               bool odd = false)
{
    return 128 + (size_t)nbuf * rowbulk_stage_elems(rowbulk_stage_rows(TR, k2, aligned), L, odd) * 4 +
           (size_t)TR * LSW * 4 + 16;
}

// Window walk of one column group of CW adjacent elements over output rows
// [s0, s1) of a tile: reads the staging buffer (rows L apart, unswizzled),
// writes the swizzled row buffer W (rows LSW apart).
//
// FULL (k == KMAX, s1 - s0 a multiple of k): blocks of k rows, each output
// the suffix of its block from the row on plus the prefix of the next block
// up to the row before its window ends -- 3k - 4 operations per column and
// block, every load and store unconditional; rows up to s1 + k - 2 are read.
// Otherwise the generic walk with runtime k <= KMAX (identity padding).
template <class M, int KMAX, int CW, bool FULL>
__device__ __forceinline__ void rowbulk_walk(const typename M::loc_t *__restrict__ st,
                                             typename M::loc_t *__restrict__ W, int L, int LSW, int c0,
                                             int s0, int s1, int k)
{
    using Lt = typename M::loc_t;
    using V = typename std::conditional<CW == 4, uint4, typename std::conditional<CW == 2, uint2, uint32_t>::type>::type;
    const Lt *sp = st + c0;
    Lt *wp = W + tswz<Lt>(c0);
    auto ld = [&](int r, Lt *v) {
        const V w = *reinterpret_cast<const V *>(sp + r * L);
        memcpy(v, &w, sizeof(V));
    };
    auto stw = [&](int r, const Lt *v) {
        V w;
        memcpy(&w, v, sizeof(V));
        *reinterpret_cast<V *>(wp + r * LSW) = w;
    };
    if constexpr (KMAX == 1) {
        for (int r = s0; r < s1; ++r) {
            Lt v[CW];
            ld(r, v);
            stw(r, v);
        }
    } else if constexpr (FULL) {
        constexpr int K = KMAX;
        Lt cur[K][CW];
#pragma unroll
        for (int j = 0; j < K; ++j) ld(s0 + j, cur[j]);
        for (int sb = s0; sb < s1; sb += K) {
            // suffixes of the current block, in place
#pragma unroll
            for (int j = K - 2; j >= 0; --j)
#pragma unroll
                for (int c = 0; c < CW; ++c) cur[j][c] = M::lop(cur[j][c], cur[j + 1][c]);
            stw(sb, cur[0]);
            const bool more = sb + K < s1;
            Lt nx[K][CW];
#pragma unroll
            for (int j = 0; j < K - 1; ++j) ld(sb + K + j, nx[j]);
            if (more) ld(sb + 2 * K - 1, nx[K - 1]);
            Lt p[CW], o[CW];
#pragma unroll
            for (int c = 0; c < CW; ++c) {
                p[c] = nx[0][c];
                o[c] = M::lop(cur[1][c], p[c]);
            }
            stw(sb + 1, o);
#pragma unroll
            for (int j = 1; j + 1 < K; ++j) {
#pragma unroll
                for (int c = 0; c < CW; ++c) {
                    p[c] = M::lop(p[c], nx[j][c]);
                    o[c] = M::lop(cur[j + 1][c], p[c]);
                }
                stw(sb + 1 + j, o);
            }
#pragma unroll
            for (int j = 0; j < K; ++j)
#pragma unroll
                for (int c = 0; c < CW; ++c) cur[j][c] = nx[j][c];
        }
    } else {
        Lt S[KMAX][CW], v[KMAX][CW];
#pragma unroll
        for (int j = 0; j < KMAX; ++j) {
            if (j < k) {
                ld(s0 + j, v[j]);
            } else {
#pragma unroll
                for (int c = 0; c < CW; ++c) v[j][c] = M::lid();
            }
        }
#pragma unroll
        for (int c = 0; c < CW; ++c) S[KMAX - 1][c] = v[KMAX - 1][c];
#pragma unroll
        for (int j = KMAX - 2; j >= 0; --j)
#pragma unroll
            for (int c = 0; c < CW; ++c) S[j][c] = M::lop(v[j][c], S[j + 1][c]);
        for (int sb = s0; sb < s1; sb += k) {
            stw(sb, S[0]);
            const int nb = sb + k;
#pragma unroll
            for (int j = 0; j < KMAX; ++j) {
                if (j < k) {
                    ld(nb + j, v[j]);
                } else {
#pragma unroll
                    for (int c = 0; c < CW; ++c) v[j][c] = M::lid();
                }
            }
            Lt p[CW];
#pragma unroll
            for (int c = 0; c < CW; ++c) p[c] = v[0][c];
#pragma unroll
            for (int j = 0; j + 1 < KMAX; ++j) {
                Lt o[CW];
#pragma unroll
                for (int c = 0; c < CW; ++c) {
                    if (j > 0) p[c] = M::lop(p[c], v[j][c]);
                    o[c] = M::lop(S[j + 1][c], p[c]);
                }
                if (j + 1 < k && sb + 1 + j < s1) stw(sb + 1 + j, o);
            }
#pragma unroll
            for (int c = 0; c < CW; ++c) S[KMAX - 1][c] = v[KMAX - 1][c];
#pragma unroll
            for (int j = KMAX - 2; j >= 0; --j)
#pragma unroll
                for (int c = 0; c < CW; ++c) S[j][c] = M::lop(v[j][c], S[j + 1][c]);
        }
    }
}

// ---------------------------------------------------------------------------
// The kernel.  Requirements (checked by the planner): the input has the
// local type (4 bytes), 128 <= L <= 1024, L % 4 == 0 unless ODD (rows of
// any length: copies and stores realigned, see `issue` and the copy-out),
// `in` and `out` 16-byte aligned, lpr = LP / EPL a power of two in [4, 32] with LP >= L, LSW =
// LP rounded up to 32, k2 <= KMAX, TR a multiple of (NT / 32) * (32 / lpr)
// (the rows one pass of the row phase covers), ntiles < 2^31, smem =
// rowbulk_smem(...).  `aligned` (k2 == KMAX and TR a multiple of the
// walk's segments times k2) selects the bounds-free walk.  LT > 0 fixes the
// row length at compile time (then L == LT, EPL * lpr == LT, LSW == LT and
// the walk must be aligned), so that strides and offsets are immediates.
// Tile t covers rows [a, a + TR) of slice t / ntile, a = (t % ntile) * TR;
// a block advances its tile coordinates without dividing.  One lane waits
// for each copy (suspending, bounded); a block barrier releases the others.
// A block that gives up waiting counts itself in g_wait_timeouts and
// returns (never expected).
// ---------------------------------------------------------------------------
template <class M, class SOut, int KMAX, int EPL, int NBUF, int NT, int LT, bool ODD = false>
__device__ __forceinline__ bool
k_rowx_bulk_body(const typename M::loc_t *__restrict__ in, const typename M::car_t *__restrict__ T,
                 SOut *__restrict__ out, int ntiles, int ntile, int n2, int L_, int k2, int k3, int TR,
                 int LSW_, int lpr_, int aligned, int64_t vbid, int64_t vgrid)
{
    const int L = LT > 0 ? LT : L_;
    const int LSW = LT > 0 ? LT : LSW_;
    const int lpr = LT > 0 ? LT / EPL : lpr_;
    using Lt = typename M::loc_t;
    using A = typename M::acc_t;
    static_assert(sizeof(Lt) == 4 && sizeof(SOut) == 4, "4-byte local and output types");
    static_assert(!ODD || LT == 0, "odd rows have a run-time length");
    constexpr int CW = rowbulk_cw(KMAX, ODD);
    constexpr int NW = NT / 32;
    extern __shared__ __align__(128) unsigned char rb_smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(rb_smem);
    const bool al = LT > 0 || aligned != 0;
    const int RSA = rowbulk_stage_rows(TR, k2, al);
    const int SB = rowbulk_stage_elems(RSA, L, ODD);   // elements per staging buffer
    Lt *stage0 = reinterpret_cast<Lt *>(rb_smem + 128);
    Lt *W = stage0 + NBUF * SB;
    Lt *idc = W + TR * LSW;   // 4 identity elements
    const int LP = lpr * EPL;
    const int rpw = 32 / lpr;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint64_t pol_in = l2_policy_evict_first();
    const uint64_t pol_out = l2_policy_evict_first();
    const int halo = k2 > 1 ? k2 - 1 : 0;
    const int grid = (int)vgrid;
    const int bid = (int)vbid;

    // ---- one-time set-up: identity that no tile overwrites ----
    if (tid < 4) idc[tid] = M::lid();
    // W: columns [L, LP) of every row (strip padding of the row phase;
    // none when the row length is fixed at compile time)
    if constexpr (LT == 0) {
        if (LP > L) {
            const int padw = LP - L;
            for (int i = tid; i < TR * padw; i += NT) {
                const int r = i / padw;
                W[r * LSW + tswz<Lt>(L + (i - r * padw))] = M::lid();
            }
        }
    }
    // staging rows past the halo (read by the walk, never copied into; odd
    // rows: filled with each tile, at its shift)
    if constexpr (!ODD)
        for (int b = 0; b < NBUF; ++b)
            for (int i = tid; i < (RSA - (TR + halo)) * L; i += NT) stage0[b * SB + (TR + halo) * L + i] = M::lid();

    // Column groups and row segments of the walk, fixed for the kernel.
    // (aligned walk: the planner's segments of whole k2-blocks; generic
    // walk: segments of at least 2 k2 rows, so that a segment's look-ahead
    // does not dominate what it reads)
    const int LQ = L / CW;
    int G = LQ >= NT ? 1 : NT / LQ;
    if (!al && k2 > 1) G = max(1, min(G, TR / (2 * k2)));
    const int SL = (TR + G - 1) / G;
    constexpr int NP = 4 / CW;   // (column group, segment) pairs per thread for L <= 1024, NT >= 256
    int pc[NP], ps[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const int cg = tid + p * NT;
        if (cg < LQ * G) {
            ps[p] = cg / LQ;
            pc[p] = (cg - ps[p] * LQ) * CW;
        } else {
            ps[p] = -1;
            pc[p] = 0;
        }
    }

    // Stages tile t into buffer b: identity in rows [nst, TR + halo) first
    // (all threads; ordered before the walk by the barriers in between),
    // then one bulk copy by thread 0.
    // Odd rows: the tile's first element lies at element offset sh (0 .. 3)
    // of the buffer, so that the copy starts on a 16-byte boundary of the
    // input; the copy ends on the last such boundary inside the tile, and
    // the at most 3 elements after it are loaded by plain loads.
    auto issue = [&](int o, int a, int b) {
        const int nst = min(TR + halo, n2 - a);
        Lt *st = stage0 + b * SB;
        const int64_t e0g = ((int64_t)o * n2 + a) * (int64_t)L;
        if constexpr (ODD) {
            const int sh = (int)(e0g & 3);
            const int64_t e1g = e0g + (int64_t)nst * L;
            const int64_t g0 = e0g - sh, gend = e1g & ~(int64_t)3;
            for (int i = tid; i < (RSA - nst) * L; i += NT) st[sh + nst * L + i] = M::lid();
            if (tid < (int)(e1g - gend)) st[(int)(gend - g0) + tid] = in[gend + tid];
            if (tid == 0) {
                fence_proxy_async_smem();
                const unsigned bytes = gend > g0 ? (unsigned)(gend - g0) * 4u : 0u;
                mbar_arrive_expect_tx(bar + b, bytes);
                if (bytes) bulk_g2s(st, in + g0, bytes, bar + b, pol_in);
            }
        } else {
            for (int i = tid; i < (TR + halo - nst) * L; i += NT) st[nst * L + i] = M::lid();
            if (tid == 0) {
                fence_proxy_async_smem();
                const unsigned bytes = (unsigned)nst * (unsigned)L * 4u;
                mbar_arrive_expect_tx(bar + b, bytes);
                bulk_g2s(st, in + e0g, bytes, bar + b, pol_in);
            }
        }
    };

    if (tid == 0) {
        for (int b = 0; b < NBUF; ++b) mbar_init(bar + b, 1);
        mbar_fence_init();
    }
    // Everything above is private set-up; the input and T may come from the
    // kernels before this one (programmatic dependent launch).
    pdl_wait();
    __syncthreads();
    // tile coordinates (slice, tile in slice) of this block's current tile
    // and of the next tile to stage; a step of `grid` tiles is (go, gj)
    const int go = grid / ntile, gj = grid - go * ntile;
    int o_cur = bid / ntile;
    int j_cur = bid - o_cur * ntile;
    int o_nx = o_cur, j_nx = j_cur;
    auto step = [&](int &oo, int &jj) {
        oo += go;
        jj += gj;
        if (jj >= ntile) {
            jj -= ntile;
            ++oo;
        }
    };
    for (int b = 0; b < NBUF; ++b) {
        if (bid + b * grid < ntiles) issue(o_nx, j_nx * TR, b);
        step(o_nx, j_nx);
    }

    // Row-phase constants: lane `sub` of a row owns strip [e0, e0 + EPL).
    const int sub = lane & (lpr - 1);
    const int rw = lane / lpr;
    const int e0 = sub * EPL;
    int toff[EPL / 4];
#pragma unroll
    for (int i = 0; i < EPL / 4; ++i) toff[i] = tswz<Lt>(e0 + 4 * i);
    const bool vsb = (k3 & 3) == 0;
    const int L4 = L >> 2;
    // shifted-suffix chunk of strip chunk i: e0 + 4 i + k3 (vector path),
    // -1 past the row end (identity)
    int soff[EPL / 4];
#pragma unroll
    for (int i = 0; i < EPL / 4; ++i) {
        const int js = e0 + 4 * i + k3;
        soff[i] = js < L ? tswz<Lt>(js) : -1;
    }
    // copy-out: lane reads chunk c = lane + 32 j of a row; its swizzled
    // offset is 128 j + 4 (lane ^ ((lane >> 3) + 4 (j & 1)))
    const int coff_e = 4 * (lane ^ (lane >> 3));
    const int coff_o = 4 * (lane ^ ((lane >> 3) + 4));

    int it = 0;
    for (int t = bid; t < ntiles; t += grid, ++it, step(o_cur, j_cur)) {
        const int b = NBUF == 1 ? 0 : it % NBUF;
        const unsigned parity = (unsigned)(it / NBUF) & 1u;
        const int o = o_cur;
        const int a = j_cur * TR;
        const int nout = min(TR, n2 - a);
        const Lt *stage = stage0 + b * SB;
        if constexpr (ODD) stage += (int)((((int64_t)o * n2 + a) * (int64_t)L) & 3);
        int ok = 1;
        if (tid == 0) ok = mbar_wait_bounded(bar + b, parity) ? 1 : 0;
        if (!__syncthreads_and(ok)) {
            if (tid == 0) atomicAdd(&g_wait_timeouts, 1u);
            return false;
        }
        // ---- window along n2: stage -> W ----
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            if (ps[p] >= 0) {
                const int s0 = ps[p] * SL;
                if (al) {
                    if (s0 < nout) rowbulk_walk<M, KMAX, CW, true>(stage, W, L, LSW, pc[p], s0, s0 + SL, k2);
                } else {
                    const int s1 = min(s0 + SL, nout);
                    if (s0 < s1) rowbulk_walk<M, KMAX, CW, false>(stage, W, L, LSW, pc[p], s0, s1, k2);
                }
            }
        }
        __syncthreads();
        // the staging buffer is free: stage a later tile under the row phase
        if (t + NBUF * grid < ntiles) issue(o_nx, j_nx * TR, b);
        step(o_nx, j_nx);

        // ---- rows: T (+) exclusive prefix (+) suffix from x_d + k3 ----
        const int64_t rowbase = (int64_t)o * n2 + a;
        for (int rb = warp * rpw; rb < nout; rb += NW * rpw) {
            // rows r >= nout (last tile of a slice) are computed on stale
            // W rows below TR and never copied out
            const int r = rb + rw;
            const bool live = r < nout;
            Lt *row = W + r * LSW;
            const A tv = live ? M::get(T[rowbase + r]) : M::id();
            Lt v[EPL];
#pragma unroll
            for (int i = 0; i < EPL / 4; ++i) {
                const uint4 w = *reinterpret_cast<const uint4 *>(row + toff[i]);
                memcpy(v + 4 * i, &w, 16);
            }
            Lt tsum = v[0];
#pragma unroll
            for (int j = 1; j < EPL; ++j) tsum = M::lop(tsum, v[j]);
            // segmented inclusive scans of the strip totals, both directions
            Lt pr = tsum, s = tsum;
#pragma unroll
            for (int lv = 0; lv < 5; ++lv) {
                const int dl = 1 << lv;
                if (dl < lpr) {
                    const Lt u = shfl_up(pr, dl);
                    const Lt w = shfl_down(s, dl);
                    if (sub >= dl) pr = M::lop(u, pr);
                    if (sub + dl < lpr) s = M::lop(s, w);
                }
            }
            pr = shfl_up(pr, 1);
            s = shfl_down(s, 1);
            if (sub == 0) pr = M::lid();
            if (sub == lpr - 1) s = M::lid();
            // inclusive suffixes of the strip, written over the strip in W
            // (only this lane read these positions)
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
                *reinterpret_cast<uint4 *>(row + toff[i]) = w;
            }
            __syncwarp();
            // results: T (+) prefix before x (+) suffix from x + k3
            Lt res[EPL];
            if (vsb) {
#pragma unroll
                for (int i = 0; i < EPL / 4; ++i) {
                    const Lt *q = soff[i] >= 0 ? row + soff[i] : idc;
                    const uint4 w = *reinterpret_cast<const uint4 *>(q);
                    Lt sv[4];
                    memcpy(sv, &w, 16);
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        res[4 * i + m] = M::lop(pr, sv[m]);
                        pr = M::lop(pr, v[4 * i + m]);
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < EPL; ++j) {
                    const int js = e0 + j + k3;
                    res[j] = M::lop(pr, js < L ? row[tswz<Lt>(js)] : M::lid());
                    pr = M::lop(pr, v[j]);
                }
            }
            __syncwarp();
            // results over the strip, in place -- never into the padding
            // columns [L, LP), which must keep the identity for later tiles
#pragma unroll
            for (int i = 0; i < EPL / 4; ++i) {
                SOut o4[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) o4[m] = finish<M, SOut>(tv, res[4 * i + m]);
                uint4 w;
                memcpy(&w, o4, 16);
                if (LP == L || e0 + 4 * i + 4 <= L) {
                    *reinterpret_cast<uint4 *>(row + toff[i]) = w;
                } else if (ODD && e0 + 4 * i < L) {
                    // the chunk holding the row's end: its columns past L stay identity
#pragma unroll
                    for (int m = 0; m < 4; ++m)
                        if (e0 + 4 * i + m < L) row[toff[i] + m] = o4[m];
                }
            }
            __syncwarp();
            if constexpr (ODD) {
                // the warp's rows are one contiguous run of the output, which
                // starts at any alignment: its whole 16-byte chunks with
                // 16-byte stores, the at most 3 elements before and after
                // them with plain ones
                const int q = min(rpw, nout - rb);
                const int64_t F0 = (rowbase + rb) * (int64_t)L, F1 = F0 + (int64_t)q * L;
                const int64_t G0 = min(F1, (F0 + 3) & ~(int64_t)3), G1 = max(G0, F1 & ~(int64_t)3);
                // (W holds the results' bits)
                auto wv = [&](int rel) {
                    const int rr = rel / L;
                    SOut v;
                    memcpy(&v, W + (rb + rr) * LSW + tswz<Lt>(rel - rr * L), 4);
                    return v;
                };
                if (lane < (int)(G0 - F0)) st_hint(out + F0 + lane, wv(lane), pol_out);
                if (lane < (int)(F1 - G1)) st_hint(out + G1 + lane, wv((int)(G1 - F0) + lane), pol_out);
                for (int64_t f = G0 + 4 * lane; f < G1; f += 128) {
                    const int rel = (int)(f - F0);
                    int rr = rel / L, cc = rel - rr * L;
                    Lt o4[4];
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        o4[m] = W[(rb + rr) * LSW + tswz<Lt>(cc)];
                        if (++cc == L) {
                            cc = 0;
                            ++rr;
                        }
                    }
                    uint4 w;
                    memcpy(&w, o4, 16);
                    st_hint_v4(out + f, w, pol_out);
                }
            } else
            // coalesced copy-out of this warp's rows
            for (int q = 0; q < rpw; ++q) {
                const int rr = rb + q;
                if (rr >= nout) break;
                const Lt *src = W + rr * LSW;
                SOut *dst = out + (rowbase + rr) * (int64_t)L + 4 * lane;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (lane + 32 * j < L4) {
                        const uint4 w = *reinterpret_cast<const uint4 *>(src + 128 * j + ((j & 1) ? coff_o : coff_e));
                        st_hint_v4(dst + 128 * j, w, pol_out);
                    }
                }
            }
        }
        __syncthreads();   // W is rewritten by the next tile's walk
    }
    // every copy issued was waited for: the barriers can be retired, so that
    // a later call of this body in the same block may initialise them again
    if (tid == 0)
        for (int b = 0; b < NBUF; ++b) mbar_inval(bar + b);
    return true;
}

template <class M, class SOut, int KMAX, int EPL, int NBUF, int NT, int LT, bool ODD = false>
__global__ void __launch_bounds__(NT, 512 / NT)
k_rowx_bulk(const typename M::loc_t *__restrict__ in, const typename M::car_t *__restrict__ T,
            SOut *__restrict__ out, int ntiles, int ntile, int n2, int L_, int k2, int k3, int TR,
            int LSW_, int lpr_, int aligned)
{
    k_rowx_bulk_body<M, SOut, KMAX, EPL, NBUF, NT, LT, ODD>(in, T, out, ntiles, ntile, n2, L_, k2, k3, TR, LSW_,
                                                          lpr_, aligned, blockIdx.x, gridDim.x);
}

}  // namespace exsum
