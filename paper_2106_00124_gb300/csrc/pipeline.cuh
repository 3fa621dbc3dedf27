// pipeline.cuh -- pass sequences of BDBS (included sums) and box-complement
// (excluded sums) for one monoid, on one CUDA stream.
//
// The same code runs in two modes: a dry run that only measures the
// workspace, and a real run that carves the workspace identically and
// launches the kernels.  Keeping both in one function keeps the workspace
// figure and the launches in step.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <type_traits>

#include "kernels_flat.cuh"
#include "kernels_fold.cuh"
#include "kernels_line1d.cuh"
#include "kernels_longrow.cuh"
#include "kernels_rowbulk.cuh"
#include "kernels_rows.cuh"

namespace exsum {

// Status codes, mirrored from include/exsum.h (kept numerically identical).
enum { ST_OK = 0, ST_EINVAL = -1, ST_ENOMEM = -2, ST_EUNSUP = -3, ST_ECUDA = -4 };

// Kernel tags reported by the launch trace (exsum_trace_*).
enum KernelTag {
    TAG_INC = 0,          // BDBS-Along-Dim, generic line pass (k > 32)
    TAG_REDUCE = 1,       // segment / column reductions
    TAG_SUMSEG = 2,       // (unused; kept so that tag numbers stay stable)
    TAG_CARRY = 3,        // dimension-1 carries
    TAG_EXLINE = 4,       // dimension-1 prefix/suffix + contributions
    TAG_INC_CONTIG = 5,   // BDBS-Along-Dim, contiguous dimension (k_inc_flat)
    TAG_INC_STRIDED = 6,  // BDBS-Along-Dim, strided dimension (k_inc_strided)
    TAG_ROWSUM = 7,       // row totals over the last dimension (k_row_totals)
    TAG_ROWX = 8,         // last-dimension prefix/suffix + contributions (k_rowx)
    TAG_WEAK = 9,         // weak excluded sums: total, then total minus included
    TAG_INC_FOLD = 10,    // BDBS-Along-Dim, strided, with partial row totals (k_inc_strided4_rt)
    TAG_PLANE = 11,       // plane totals of the two-dimensional lower problem (k_plane_totals)
    TAG_EXC2D = 12,       // excluded sums of the two-dimensional lower problem (k_exc2d)
    TAG_COUNT = 13
};

// Launch bracketing for the trace and the launch counter (exsum_abi.cu).
void trace_before(cudaStream_t s, int tag, int level, int64_t elems);
void trace_after(cudaStream_t s);

// Side stream and fork/join events for running independent passes
// concurrently with the caller's stream (a parallel branch under capture).
struct Aux {
    cudaStream_t side = nullptr, side2 = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, fork2 = nullptr, join2 = nullptr;
};

struct Ctx {
    const Aux *aux = nullptr;    // nullptr: everything on `stream`
    char *base = nullptr;   // workspace (device)
    size_t cap = 0;         // workspace bytes available
    size_t off = 0;         // bytes carved so far
    bool dry = true;        // measure only
    cudaStream_t stream = 0;
    int status = ST_OK;
    cudaError_t cuda_err = cudaSuccess;
    int level = 0;           // recursion depth of box-complement (0 = input tensor)
    int64_t sms = 152;       // streaming multiprocessors of the device

    template <class T>
    T *take(int64_t count)
    {
        const size_t bytes = ((size_t)count * sizeof(T) + 255) & ~(size_t)255;
        T *p = dry ? nullptr : reinterpret_cast<T *>(base + off);
        off += bytes;
        if (!dry && off > cap && status == ST_OK) status = ST_ENOMEM;
        return p;
    }
    bool ok() const { return status == ST_OK; }
    void before(int tag, int64_t elems) { trace_before(stream, tag, level, elems); }
    void check_launch()
    {
        if (dry) return;
        trace_after(stream);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess && status == ST_OK) {
            status = ST_ECUDA;
            cuda_err = e;
        }
    }
};

static inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Launches `kern` on `stream` with programmatic stream serialization: it may
// start while the kernel before it on the stream finishes, and waits for it
// with pdl_wait() before touching that kernel's results.  Launch latency of
// a chain of short dependent kernels is hidden this way.
template <class... KArgs, class... Args>
static inline void launch_pdl(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem,
                              cudaStream_t stream, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, (KArgs)args...);
}

// Streaming multiprocessors of the current device, looked up once per device
// (grids and tile heights are sized by it).  Without a usable device (a
// workspace query on a machine with no GPU) the GB300's 152 is assumed.
inline int device_sms()
{
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 152;
    }
    if (cache[dev] <= 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            v = 152;
        }
        cache[dev] = v;
    }
    return cache[dev];
}

template <class M>
struct Pipe {
    // Monoid for work on carries (compensated local arithmetic for fp +).
    using MC = typename std::conditional<M::compensated, MonComp<M>, M>::type;
    using A = typename M::acc_t;
    using IN = typename M::in_t;
    using OUT = typename M::out_t;
    using CAR = typename M::car_t;

    static constexpr int EXL = 32;            // segment length of the dimension-1 step
    // the two-kernel lower problem combines all n_1 plane totals for each
    // plane: at most this many planes
    static constexpr int64_t SMALL2D_N1 = 16384;
    static constexpr int INC_THREADS = 128;
    static constexpr size_t SLOT_SMEM_MAX = 96 * 1024;

    // ---- BDBS-Along-Dim over a view [O, n, I] -------------------------------------
    using L_ = typename M::loc_t;
    static constexpr int CONTIG_ROWS = sizeof(L_) > 4 ? 64 : 128;

    // Rsum/Rtail (contiguous pass only): also produce the segment totals of the
    // input over the view's first dimension n1 (segments of EXL rows).
    template <class SIn, class SOut, int KMAX>
    static void inc_fast(Ctx &cx, const SIn *src, SOut *dst, int64_t O, int64_t n, int64_t I,
                         int64_t k, int64_t n1 = 1, CAR *Rsum = nullptr, CAR *Rtail = nullptr,
                         int r_tail = 0)
    {
        if (I == 1) {
            // Contiguous dimension: warp chunks of 128 elements of a "plane".
            // With segment totals the planes are the slices of dimension 1;
            // otherwise a plane is a run of whole rows of at least 128 elements.
            const int64_t N = O * n;
            int64_t pn1, M1;
            if (Rsum) {
                pn1 = n1;
                M1 = N / n1;
            } else {
                const int64_t rpp = cdiv(128, n);
                M1 = rpp * n;
                pn1 = cdiv(O, rpp);
            }
            const int64_t nq = cdiv(M1, 128);
            const int64_t blocks = cdiv(pn1, 32) * nq;
            cx.before(TAG_INC_CONTIG, N);
            k_inc_flat<M, SIn, SOut, KMAX><<<(unsigned)blocks, 256, 0, cx.stream>>>(
                src, dst, N, pn1, M1, n, (int)k, nq, Rsum, Rtail, r_tail);
            cx.check_launch();
        } else {
            if constexpr (KMAX <= 8 && sizeof(L_) == 4 && sizeof(SOut) == 4) {
                if ((I & 3) == 0 && (((uintptr_t)src) & (sizeof(SIn) * 4 - 1)) == 0 &&
                    (((uintptr_t)dst) & 15) == 0) {
                    // Four inner positions per thread, 16-byte accesses;
                    // chunks short enough for ~1024 threads per SM.
                    int Lc = 128;
                    while (Lc > 2 * k && Lc > 16 && O * cdiv(n, Lc) * (I / 4) < cx.sms * 1024) Lc >>= 1;
                    if (Lc > n) Lc = (int)n;
                    const int nchunks = (int)cdiv(n, Lc);
                    const int64_t total = O * nchunks * (I / 4);
                    cx.before(TAG_INC_STRIDED, O * n * I);
                    k_inc_strided4<M, SIn, SOut, KMAX><<<(unsigned)cdiv(total, 128), 128, 0, cx.stream>>>(
                        src, dst, O, (int)n, I, (int)k, Lc, nchunks);
                    cx.check_launch();
                    return;
                }
            }
            // Chunks short enough for ~2048 threads per SM (walks of a few blocks).
            int Lc = 128;
            while (Lc > 2 * k && Lc > 16 && O * cdiv(n, Lc) * I < cx.sms * 2048) Lc >>= 1;
            if (Lc > n) Lc = (int)n;
            const int nchunks = (int)cdiv(n, Lc);
            const int64_t total = O * nchunks * I;
            cx.before(TAG_INC_STRIDED, O * n * I);
            k_inc_strided<M, SIn, SOut, KMAX><<<(unsigned)cdiv(total, 128), 128, 0, cx.stream>>>(
                src, dst, O, (int)n, I, (int)k, Lc, nchunks);
            cx.check_launch();
        }
    }

    template <class SIn, class SOut>
    static void inc_pass(Ctx &cx, const SIn *src, SOut *dst, int64_t O, int64_t n, int64_t I,
                         int64_t k)
    {
        if (!cx.ok()) return;
        if (k <= 32 && n < (1ll << 30)) {
            if (cx.dry) return;
            if (k <= 4)
                inc_fast<SIn, SOut, 4>(cx, src, dst, O, n, I, k);
            else if (k <= 8)
                inc_fast<SIn, SOut, 8>(cx, src, dst, O, n, I, k);
            else if (k <= 16)
                inc_fast<SIn, SOut, 16>(cx, src, dst, O, n, I, k);
            else
                inc_fast<SIn, SOut, 32>(cx, src, dst, O, n, I, k);
            return;
        }
        // Large boxes along a strided dimension: one block of k lines per
        // thread, the block's suffixes kept in the output (k_inc_strided_big).
        if (I > 1 && n < (1ll << 30) && env_int("EXSUM_BIGK", 1) != 0) {
            if (cx.dry) return;
            const int64_t nchunks = cdiv(n, k);
            const int64_t total = O * nchunks * I;
            cx.before(TAG_INC_STRIDED, O * n * I);
            k_inc_strided_big<M, SIn, SOut><<<(unsigned)cdiv(total, 128), 128, 0, cx.stream>>>(
                src, dst, O, (int)n, I, (int)k, (int)k, (int)nchunks);
            cx.check_launch();
            return;
        }
        // Large boxes along the contiguous dimension: one warp per segment of
        // whole blocks of a row (k_inc_rows_big).
        if (I == 1 && env_int("EXSUM_BIGK", 1) != 0) {
            if (cx.dry) return;
            const int64_t G = k * (k < 1024 ? 1024 / k : 1);
            const int64_t nseg = cdiv(n, G);
            const int64_t warps = O * nseg;
            cx.before(TAG_INC_CONTIG, O * n);
            k_inc_rows_big<M, SIn, SOut><<<(unsigned)cdiv(warps * 32, 256), 256, 0, cx.stream>>>(
                src, dst, O, n, k, G, nseg);
            cx.check_launch();
            return;
        }
        // Otherwise: per-thread suffix slots in shared or global memory.
        int threads = INC_THREADS;
        while (threads > 32 && (size_t)k * threads * sizeof(A) > SLOT_SMEM_MAX) threads >>= 1;
        const bool global_slots = (size_t)k * threads * sizeof(A) > SLOT_SMEM_MAX;
        int64_t Lc = 64 > 2 * k ? 64 : 2 * k;
        if (global_slots && Lc < 4 * k) Lc = 4 * k;
        if (Lc > n) Lc = n;
        const int64_t nchunks = cdiv(n, Lc);
        const int64_t total = O * nchunks * I;
        A *gslots = global_slots ? cx.take<A>(total * k) : nullptr;
        if (cx.dry || !cx.ok()) return;
        const size_t smem = global_slots ? 0 : (size_t)k * threads * sizeof(A);
        auto kern = k_inc_lines<M, SIn, SOut>;
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cx.before(TAG_INC, O * n * I);
        kern<<<(unsigned)cdiv(total, threads), threads, smem, cx.stream>>>(src, dst, O, n, I, k, Lc,
                                                                           nchunks, gslots);
        cx.check_launch();
    }

    // ---- dimension-1 step: prefix/suffix along dim 1 + contributions --------------------
    static constexpr int CT_NT = 256, CT_V = 16, CT_L = CT_NT * CT_V;  // contiguous segment
    static constexpr int LN_NT = 256, LN_V = 16, LN_L = LN_NT * LN_V;  // one long line, 16-byte path

    template <class SH, class SOut>
    static void exline_stage(Ctx &cx, const SH *H, const CAR *T, SOut *out, int64_t n1,
                             int64_t Mc, int64_t k1)
    {
        if (!cx.ok()) return;
        const bool contig = (Mc == 1);
        // one long line with a 4-byte local type: 16-byte loads and stores
        // (kernels_line1d.cuh)
        const bool line = contig && sizeof(L_) == 4 && T == nullptr;
        const int64_t L = line ? LN_L : (contig ? CT_L : EXL);
        const int64_t S = cdiv(n1, L);
        const CAR *Q = T;
        int64_t qs = 0;
        if (S > 1) {
            CAR *R = cx.take<CAR>(S * Mc);
            CAR *Rt = cx.take<CAR>(S * Mc);
            CAR *Qb = cx.take<CAR>(S * Mc);
            const bool blk = S > 64 && Mc < 4096;
            CAR *SR = blk ? cx.take<CAR>(S * Mc) : nullptr;
            if (cx.dry || !cx.ok()) return;
            const int64_t qoff = 1 + k1 / L;
            if (line) {
                const int vec = ((((uintptr_t)H) & (sizeof(SH) * 4 - 1)) == 0) ? 1 : 0;
                cx.before(TAG_REDUCE, n1);
                k_reduce_line<M, SH, LN_NT, LN_V><<<(unsigned)S, LN_NT, 0, cx.stream>>>(H, R, Rt, n1, k1 % L, vec);
                cx.check_launch();
                cx.before(TAG_CARRY, S);
                k_carry_line2<M, 1024><<<(unsigned)cdiv(S, 1024), 1024, 0, cx.stream>>>(R, Rt, Qb, S, qoff);
                cx.check_launch();
            } else {
                cx.before(TAG_REDUCE, n1 * Mc);
                if (contig)
                    k_reduce_seg_contig<M, SH, CT_NT, CT_V><<<(unsigned)S, CT_NT, 0, cx.stream>>>(
                        H, R, Rt, n1, k1 % L);
                else
                    k_reduce_seg2<M, SH><<<(unsigned)cdiv(S * Mc, 256), 256, 0, cx.stream>>>(
                        H, R, Rt, n1, Mc, L, S, k1 % L);
                cx.check_launch();
                cx.before(TAG_CARRY, S * Mc);
                if (blk)
                    k_carry_blk<M, 1024><<<(unsigned)Mc, 1024, 0, cx.stream>>>(R, Rt, T, Qb, SR, Mc, S,
                                                                               qoff, nullptr);
                else
                    k_carry_col<M><<<(unsigned)cdiv(Mc, 256), 256, 0, cx.stream>>>(R, Rt, T, Qb, Mc, S,
                                                                                    qoff);
                cx.check_launch();
            }
            Q = Qb;
            qs = Mc;
        }
        if (cx.dry || !cx.ok()) return;
        cx.before(TAG_EXLINE, n1 * Mc);
        if (line) {
            const int vin = ((((uintptr_t)H) & (sizeof(SH) * 4 - 1)) == 0) ? 1 : 0;
            const int vout = ((((uintptr_t)out) & 15) == 0 && sizeof(SOut) == 4) ? 1 : 0;
            k_exline_line<M, SH, SOut, LN_NT, LN_V><<<(unsigned)S, LN_NT, 0, cx.stream>>>(
                H, Q, out, n1, k1, vin, vin && (k1 % 4) == 0 ? 1 : 0, vout);
        } else if (contig) {
            k_exline_contig<M, SH, SOut, CT_NT, CT_V><<<(unsigned)S, CT_NT, 0, cx.stream>>>(
                H, Q, out, n1, k1);
        } else {
            k_exline2<M, SH, SOut, EXL><<<(unsigned)cdiv(S * Mc, 128), 128, 0, cx.stream>>>(
                H, Q, qs, nullptr, out, n1, Mc, k1, S);
        }
        cx.check_launch();
    }

    // Dimension-1 step over a view [n1, Mc], Mc > 1: rows staged in shared
    // memory by asynchronous copies when the element is 4 or 8 bytes wide.
    template <class SH, class SOut>
    static void exline_launch(Ctx &cx, const SH *H, const CAR *Q, const CAR *T, SOut *out,
                              int64_t n1, int64_t Mc, int64_t k1, int64_t S)
    {
        k_exline2<M, SH, SOut, EXL><<<(unsigned)cdiv(S * Mc, 128), 128, 0, cx.stream>>>(
            H, Q, Mc, T, out, n1, Mc, k1, S);
    }

    // ---- included sums: BDBS along every dimension ---------------------------------------
    template <class SIn, class SOut>
    static void included(Ctx &cx, const SIn *X, SOut *out, int d, const int64_t *n,
                         const int64_t *k)
    {
        int64_t N = 1;
        for (int i = 0; i < d; ++i) N *= n[i];
        int dims[16];
        int P = 0;
        for (int j = d - 1; j >= 0; --j)
            if (k[j] > 1) dims[P++] = j;
        if (P == 0) dims[P++] = d - 1;  // a k = 1 pass converts the input type
        SOut *B = P > 1 ? cx.take<SOut>(N) : nullptr;
        const void *cur = X;
        for (int p = 0; p < P; ++p) {
            const int j = dims[p];
            int64_t O = 1, I = 1;
            for (int m = 0; m < j; ++m) O *= n[m];
            for (int m = j + 1; m < d; ++m) I *= n[m];
            SOut *dst = ((P - 1 - p) % 2 == 0) ? out : B;
            if (p == 0)
                inc_pass<SIn, SOut>(cx, (const SIn *)cur, dst, O, n[j], I, k[j]);
            else
                inc_pass<SOut, SOut>(cx, (const SOut *)cur, dst, O, n[j], I, k[j]);
            cur = dst;
        }
    }

    // ---- excluded sums with the last dimension peeled (kernels_rows.cuh) ---------------------
    //
    // Level with input X of shape n[0..d-1], L = n[d-1]:
    //   R  = total of X over dimension d                          (dimension reduction)
    //   T  = excluded sum of R with box k[0..d-2]                 (next level)
    //   H  = included sum of X along dimensions 1..d-1            (BDBS-Along-Dim)
    //   out[x] = T[x_1..x_{d-1}] (+) prefix of H's row before x_d (+) suffix of the row from x_d+k_d
    // The rows are short enough for one warp to scan a row from shared memory,
    // so this needs no carries; the window along dimension d-1 is fused into
    // the final pass when its tile holds enough rows.
    static constexpr int ROWX_THREADS = 256;
    static constexpr int64_t ROWX_TAIL = 4096;  // 1-D recursion folded into the final pass

    struct RowPlan {
        bool ok = false, fuse = false, longrow = false;
        int GO = 1, TR = 1, ntile = 1, RS = 1, RSA = 1, LS = 16, lpr = 32, epl = 4;
        size_t smem = 0;
    };

    static int row_lanes(int64_t L)
    {
        const int64_t q4 = cdiv(L, 4);
        int lpr = 1;
        while (lpr < q4 && lpr < 32) lpr <<= 1;
        return lpr;
    }

    // Tile geometry of the final pass: GO slices x TR rows per block.  The
    // window along n_{d-1} is fused when the staged halo (k2 - 1 rows) is at
    // most about half the tile, or the tile is the whole slice; small tensors
    // get shorter tiles (more blocks) down to that limit.
    static RowPlan row_plan(int d, const int64_t *n, const int64_t *k, int64_t sms)
    {
        RowPlan rp;
        if (d < 2) return rp;
        const int64_t L = n[d - 1];
        const int64_t s = (int64_t)sizeof(L_);
        const int64_t lmax = s > 4 ? 512 : 1024;
        if (L < 16 || L > lmax || n[d - 2] >= (1ll << 30)) return rp;
        int64_t O2 = 1;
        for (int m = 0; m < d - 2; ++m) O2 *= n[m];
        const int64_t n2 = n[d - 2], k2 = k[d - 2];
        const int64_t CE = 16 / s;
        const int64_t LS = cdiv(L, 8 * CE) * 8 * CE;
        const int64_t L32 = cdiv(L, 32) * 32;
        const int64_t LPs = L32 + 4 * (L32 / 32) + 4;
        const int64_t lpr = row_lanes(L);
        int64_t epl = 4;   // 4, 8, 16 or 32 elements per lane
        while (epl * lpr < L) epl <<= 1;
        const int64_t rpw = 32 / lpr;
        int64_t GO = ROWX_THREADS / L;
        if (GO < 1) GO = 1;
        if (GO > O2) GO = O2;
        const int64_t groups = cdiv(O2, GO);
        // rows per tile for at least two blocks per SM, when the tensor has them
        const int64_t tr_par = groups >= 2 * sms ? n2 : cdiv(n2, cdiv(2 * sms, groups));
        // rows a tile holds: TR, the k2 - 1 halo rows and the identity rows the
        // column walk may read past them
        auto rows_held = [&](int64_t tr, bool f) -> int64_t {
            return f ? (tr - 1) / k2 * k2 + 2 * k2 : tr;
        };
        auto fit = [&](int64_t budget, bool f, int64_t &TR, int64_t &ntile) -> bool {
            int64_t tr = f ? (tr_par > 2 * k2 ? tr_par : 2 * k2) : tr_par;
            if (tr > 64) tr = 64;
            while (tr >= 1 && rows_held(tr, f) * GO * LS * s > budget) --tr;
            if (tr < 1) return false;
            if (tr >= 16) tr &= ~(int64_t)7;
            ntile = cdiv(n2, tr);
            TR = cdiv(n2, ntile);
            return !f || ntile == 1 || TR >= 2 * k2;
        };
        int64_t TR = 1, ntile = 1;
        bool fuse = false;
        // Four blocks per SM (228 KB, 1 KB reserved per block, less the
        // suffix rows and T) when that still gives tiles of at least 32 rows
        // or whole slices; otherwise the tallest tile (at most 64 rows) two
        // blocks per SM allow, so that the halo rows stay a small part of
        // what a block stages.
        const int64_t extra = (int64_t)(ROWX_THREADS / 32) * rpw * LPs * s + 2 * 64 * 16 + 64 * 16;
        const int64_t four = 56 * 1024 - extra, two = 113 * 1024 - extra;
        if (k2 > 1 && k2 <= 32) {
            fuse = fit(four, true, TR, ntile) && (ntile == 1 || TR >= 32);
            if (!fuse) fuse = fit(two, true, TR, ntile);
        }
        if (!fuse && !fit(four, false, TR, ntile)) return rp;
        if (groups * ntile >= (1ll << 31)) return rp;
        rp.ok = true;
        rp.fuse = fuse;
        rp.GO = (int)GO;
        rp.TR = (int)TR;
        rp.ntile = (int)ntile;
        rp.RS = (int)(fuse ? TR + k2 - 1 : TR);
        rp.RSA = (int)rows_held(TR, fuse);
        rp.LS = (int)LS;
        rp.lpr = (int)lpr;
        rp.epl = (int)epl;
        rp.smem = ((size_t)(GO * rp.RSA * LS + (ROWX_THREADS / 32) * rpw * LPs) * s + 15) / 16 * 16 +
                  (size_t)((GO * TR > 2 * TR + 64) ? GO * TR : 2 * TR + 64) * sizeof(CAR);  // + the tile's T (and a 1-D tail's totals)
        return rp;
    }

    template <class SF, class SOut, int KM, int EPL>
    static void rowx_epl(Ctx &cx, const RowPlan &rp, const SF *src, const CAR *T, const CAR *R1,
                         SOut *out, int64_t O2, int64_t n2, int64_t L, int kk, int k3, int k1)
    {
        auto kern = k_rowx<M, SF, SOut, KM, EPL>;
        if (rp.smem > 48 * 1024)
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rp.smem);
        const unsigned blocks = (unsigned)(cdiv(O2, rp.GO) * rp.ntile);
        kern<<<blocks, ROWX_THREADS, rp.smem, cx.stream>>>(src, T, R1, k1, out, O2, (int)n2, (int)L,
                                                          kk, k3, rp.TR, rp.GO, rp.ntile, rp.RS,
                                                          rp.RSA, rp.LS, rp.lpr);
    }

    template <class SF, class SOut, int KM>
    static void rowx_go(Ctx &cx, const RowPlan &rp, const SF *src, const CAR *T, const CAR *R1, SOut *out,
                        int64_t O2, int64_t n2, int64_t L, int kk, int k3, int k1)
    {
        if (rp.epl == 4)
            rowx_epl<SF, SOut, KM, 4>(cx, rp, src, T, R1, out, O2, n2, L, kk, k3, k1);
        else if (rp.epl == 8)
            rowx_epl<SF, SOut, KM, 8>(cx, rp, src, T, R1, out, O2, n2, L, kk, k3, k1);
        else if (rp.epl == 16)
            rowx_epl<SF, SOut, KM, 16>(cx, rp, src, T, R1, out, O2, n2, L, kk, k3, k1);
        else if (rp.epl == 32 && sizeof(L_) == 4)
            rowx_epl<SF, SOut, KM, (sizeof(L_) == 4 ? 32 : 16)>(cx, rp, src, T, R1, out, O2, n2, L, kk, k3, k1);
        else if (cx.status == ST_OK)
            cx.status = ST_EUNSUP;  // not reachable: row_plan gives one of the widths above
    }

    // ---- final pass staged by bulk copies (kernels_rowbulk.cuh) ---------------------------
    struct BulkPlan {
        bool ok = false, aligned = false, pdl = false, odd = false;
        int TR = 0, epl = 32, lpr = 8, LSW = 0, nbuf = 2, nt = 256;
        size_t smem = 0;
        int ntiles = 0, grid = 0, ntile = 0;
    };

    static int env_int(const char *name, int dflt)
    {
        const char *v = getenv(name);
        return (v && *v) ? atoi(v) : dflt;
    }

    // Geometry of k_rowx_bulk for rows of L elements, a window of kk rows
    // along n2 (1: none; kmax its compile-time bound) and O2 slices of n2
    // rows: strips of 32 elements, 256 threads; two staging buffers and the
    // tallest tile (at most 64 rows, a multiple of the rows one row pass
    // covers and of the walk's segments) that lets two blocks share an SM,
    // else one staging buffer, else one block per SM.  EXSUM_ROWX_TR and
    // EXSUM_ROWX_NBUF override (tuning), and nbuf_force / tr_force override
    // those.
    static BulkPlan bulk_plan(int64_t L, int64_t n2, int64_t O2, int kk, int kmax, int64_t sms,
                              int nbuf_force = 0, int tr_force = 0)
    {
        BulkPlan bp;
        // (shorter rows stay with k_rowx: tiles of a few KB and walks over a
        // handful of columns cost more than the bulk copies save)
        if (sizeof(L_) != 4 || L < 128 || L > 1024 || kk > 32) return bp;
        const bool odd = (L & 3) != 0 && env_int("EXSUM_ROWX_ODD", 1) != 0;
        if ((L & 3) && !odd) return bp;
        // strips of 32 elements, 4 .. 32 lanes per row
        const int epl = 32;
        int lpr = 4;
        while (lpr < 32 && (int64_t)lpr * epl < L) lpr <<= 1;
        const int LP = lpr * epl;
        const int LSW = (LP + 31) & ~31;
        const int nt = 256;
        const int nb_env = nbuf_force ? nbuf_force : env_int("EXSUM_ROWX_NBUF", 0);
        const int rows_pass = (nt / 32) * (32 / lpr);
        const int G = rowbulk_segs((int)L, kmax, nt, odd);
        // block-aligned walk when the tile can be a multiple of the segments
        // times the window (at most 64 rows), else the generic walk
        bool kfull = kk > 1 && kk == kmax;
        int step = rows_pass;
        if (kfull) {
            while (step <= 64 && (step % G || (step / G) % kk)) step += rows_pass;
            if (step > 64) {
                kfull = false;
                step = rows_pass;
            }
        }
        const int tr_env = tr_force ? tr_force : env_int("EXSUM_ROWX_TR", 0);
        auto sm = [&](int tr, int nb) {
            const bool al = kfull && (tr / G) % kk == 0 && tr % G == 0;
            return rowbulk_smem(tr, kk, al, (int)L, LSW, nb, odd);
        };
        const size_t two = 113 * 1024, one = 226 * 1024;
        // candidates in order of preference: (staging buffers, blocks per SM)
        const int cand[3][2] = {{2, 2}, {1, 2}, {1, 1}};
        int TR = 0, nbuf = 1, bps = 2;
        const int trmax = step > 64 ? step : 64;
        for (int c = 0; c < 3 && !TR; ++c) {
            const int nb = cand[c][0];
            if (nb_env && nb != nb_env) continue;
            if (odd && nb != 2) continue;
            const size_t lim = cand[c][1] == 2 ? two : one;
            if (tr_env > 0) {
                const int tr = (tr_env + step - 1) / step * step;
                if (sm(tr, nb) <= lim) TR = tr;
            } else {
                for (int tr = (trmax / step) * step; tr >= step && !TR; tr -= step)
                    if (sm(tr, nb) <= lim) TR = tr;
            }
            if (TR) {
                nbuf = nb;
                bps = cand[c][1];
            }
        }
        if (!TR) return bp;
        const size_t smem = sm(TR, nbuf);
        if (smem > one) return bp;
        const int64_t ntile = cdiv(n2, TR);
        if (O2 * ntile >= (1ll << 31)) return bp;
        bp.ok = true;
        bp.aligned = kfull && (TR / G) % kk == 0 && TR % G == 0;
        bp.odd = odd;
        bp.TR = TR;
        bp.epl = epl;
        bp.lpr = lpr;
        bp.LSW = LSW;
        bp.nbuf = nbuf;
        bp.nt = nt;
        bp.smem = smem;
        bp.ntile = (int)ntile;
        bp.ntiles = (int)(O2 * ntile);
        bp.grid = (int)(bp.ntiles < sms * bps ? bp.ntiles : sms * bps);
        return bp;
    }

    template <class SOut, int KM, int EPL, int NB, int NT, int LT = 0, bool ODD = false>
    static void rowbulk_go(Ctx &cx, const BulkPlan &bp, const L_ *src, const CAR *T, SOut *out,
                           int64_t n2, int64_t L, int kk, int k3)
    {
        auto kern = k_rowx_bulk<M, SOut, KM, EPL, NB, NT, LT, ODD>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bp.smem);
        if (bp.pdl)
            launch_pdl(kern, (unsigned)bp.grid, NT, bp.smem, cx.stream, src, T, out, bp.ntiles, bp.ntile,
                       (int)n2, (int)L, kk, k3, bp.TR, bp.LSW, bp.lpr, bp.aligned ? 1 : 0);
        else
            kern<<<(unsigned)bp.grid, NT, bp.smem, cx.stream>>>(src, T, out, bp.ntiles, bp.ntile, (int)n2,
                                                                (int)L, kk, k3, bp.TR, bp.LSW, bp.lpr,
                                                                bp.aligned ? 1 : 0);
    }

    template <class SOut, int KM>
    static void rowbulk_epl(Ctx &cx, const BulkPlan &bp, const L_ *src, const CAR *T, SOut *out,
                            int64_t n2, int64_t L, int kk, int k3)
    {
        // rows of a length not a multiple of 4: two staging buffers only
        if (bp.odd) {
            rowbulk_go<SOut, KM, 32, 2, 256, 0, true>(cx, bp, src, T, out, n2, L, kk, k3);
            return;
        }
        // row lengths fixed at compile time for the common block-aligned cases
        if constexpr (KM == 4 || KM == 8) {
            if (bp.aligned && bp.LSW == L && bp.lpr * bp.epl == L) {
                if (L == 256) {
                    if (bp.nbuf == 2)
                        rowbulk_go<SOut, KM, 32, 2, 256, 256>(cx, bp, src, T, out, n2, L, kk, k3);
                    else
                        rowbulk_go<SOut, KM, 32, 1, 256, 256>(cx, bp, src, T, out, n2, L, kk, k3);
                    return;
                }
                if (L == 512) {
                    if (bp.nbuf == 2)
                        rowbulk_go<SOut, KM, 32, 2, 256, 512>(cx, bp, src, T, out, n2, L, kk, k3);
                    else
                        rowbulk_go<SOut, KM, 32, 1, 256, 512>(cx, bp, src, T, out, n2, L, kk, k3);
                    return;
                }
                if (L == 128 && bp.nbuf == 2) {
                    rowbulk_go<SOut, KM, 32, 2, 256, 128>(cx, bp, src, T, out, n2, L, kk, k3);
                    return;
                }
            }
        }
        if (bp.nbuf == 1)
            rowbulk_go<SOut, KM, 32, 1, 256>(cx, bp, src, T, out, n2, L, kk, k3);
        else
            rowbulk_go<SOut, KM, 32, 2, 256>(cx, bp, src, T, out, n2, L, kk, k3);
    }

    // Launches k_rowx_bulk when the pass qualifies (4-byte local type read
    // as is, 16-byte aligned input and output, 128 <= L <= 1024, no
    // one-dimensional tail); returns false otherwise.
    template <class SF, class SOut>
    static bool rowbulk_try(Ctx &cx, const SF *src, const CAR *T, SOut *out, int64_t O2, int64_t n2,
                            int64_t L, int kk, int k3, bool pdl = false)
    {
        if constexpr (sizeof(L_) == 4 && std::is_same<SF, L_>::value && sizeof(SOut) == 4) {
            if (env_int("EXSUM_ROWX_KERNEL", 1) == 0) return false;
            if ((((uintptr_t)src) & 15) || (((uintptr_t)out) & 15)) return false;
            const int kmax = kk <= 1 ? 1 : kk <= 4 ? 4 : kk <= 8 ? 8 : kk <= 16 ? 16 : 32;
            BulkPlan bp = bulk_plan(L, n2, O2, kk, kmax, cx.sms);
            if (!bp.ok) return false;
            bp.pdl = pdl;
            if (bp.nt != 256 || bp.epl != 32) return false;
            if (kmax == 1)
                rowbulk_epl<SOut, 1>(cx, bp, src, T, out, n2, L, 1, k3);
            else if (kmax == 4)
                rowbulk_epl<SOut, 4>(cx, bp, src, T, out, n2, L, kk, k3);
            else if (kmax == 8)
                rowbulk_epl<SOut, 8>(cx, bp, src, T, out, n2, L, kk, k3);
            else if (kmax == 16)
                rowbulk_epl<SOut, 16>(cx, bp, src, T, out, n2, L, kk, k3);
            else
                rowbulk_epl<SOut, 32>(cx, bp, src, T, out, n2, L, kk, k3);
            return true;
        } else {
            return false;
        }
    }

    // Rows longer than one warp scans (k_rowx_long, one block per row,
    // strips of 16 or 32 elements per thread -- long strips keep the block's
    // compensated scans a small part of the work per element -- in blocks
    // of 128 .. 512 threads): the row schedule without the window along
    // n_{d-1} in the final pass.  The local suffixes of a row stay in shared
    // memory: up to 16384 elements of 4 bytes, 8192 of 8.  Taken by default
    // for d = 2 and rows of at most 4096 elements, where it measured faster
    // than the dimension-1 schedule; EXSUM_LONGROW=2 takes it for every
    // shape it can hold, 0 never.
    static constexpr int LONGROW_NT = 512;
    static RowPlan long_row_plan(int d, const int64_t *n)
    {
        RowPlan rp;
        const int mode = env_int("EXSUM_LONGROW", 1);
        if (d < 2 || mode == 0) return rp;
        const int64_t L = n[d - 1];
        const int64_t lmax = sizeof(L_) > 4 ? 512 : 1024;
        const int64_t longmax = (int64_t)LONGROW_NT * (sizeof(L_) > 4 ? 16 : 32);
        if (L <= lmax || L > longmax || n[d - 2] >= (1ll << 30)) return rp;
        if (mode == 1 && (d != 2 || L > 4096)) return rp;
        rp.ok = true;
        rp.longrow = true;
        rp.fuse = false;
        return rp;
    }

    template <class SF, class SOut, int NT, int V>
    static void rowx_long_v(Ctx &cx, const SF *src, const CAR *T, SOut *out, int64_t rows, int64_t L, int k3)
    {
        auto kern = k_rowx_long<M, SF, SOut, NT, V>;
        const size_t smem = rowx_long_smem<M>(NT, V);
        if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const int64_t cap = cx.sms * (2048 / NT);
        const int64_t grid = rows < cap ? rows : cap;
        kern<<<(unsigned)grid, NT, smem, cx.stream>>>(src, T, out, rows, (int)L, k3);
    }

    template <class SF, class SOut>
    static void rowx_long_go(Ctx &cx, const SF *src, const CAR *T, SOut *out, int64_t rows, int64_t L, int k3)
    {
        if (L <= 128 * 16)
            rowx_long_v<SF, SOut, 128, 16>(cx, src, T, out, rows, L, k3);
        else if (L <= 256 * 16)
            rowx_long_v<SF, SOut, 256, 16>(cx, src, T, out, rows, L, k3);
        else if (L <= 512 * 16)
            rowx_long_v<SF, SOut, 512, 16>(cx, src, T, out, rows, L, k3);
        else if constexpr (sizeof(L_) == 4)
            rowx_long_v<SF, SOut, 512, 32>(cx, src, T, out, rows, L, k3);
    }

    template <class SF, class SOut>
    static void rowx_launch(Ctx &cx, const RowPlan &rp, const SF *src, const CAR *T, const CAR *R1, SOut *out,
                            int64_t O2, int64_t n2, int64_t L, int64_t k2, int64_t k3, bool pdl = false)
    {
        if (cx.dry || !cx.ok()) return;
        // the 1-D tail (d == 2) is the excluded sum of R along n2 with box k2
        const int k1 = R1 ? (int)k2 : 0;
        cx.before(TAG_ROWX, O2 * n2 * L);
        const int kk = rp.fuse ? (int)k2 : 1;
        if (rp.longrow) {
            rowx_long_go<SF, SOut>(cx, src, T, out, O2 * n2, L, (int)k3);
            cx.check_launch();
            return;
        }
        if (!R1 && rowbulk_try<SF, SOut>(cx, src, T, out, O2, n2, L, kk, (int)k3, pdl)) {
            cx.check_launch();
            return;
        }
        if (!rp.fuse)
            rowx_go<SF, SOut, 1>(cx, rp, src, T, R1, out, O2, n2, L, 1, (int)k3, k1);
        else if (kk <= 4)
            rowx_go<SF, SOut, 4>(cx, rp, src, T, R1, out, O2, n2, L, kk, (int)k3, k1);
        else if (kk <= 8)
            rowx_go<SF, SOut, 8>(cx, rp, src, T, R1, out, O2, n2, L, kk, (int)k3, k1);
        else if (kk <= 16)
            rowx_go<SF, SOut, 16>(cx, rp, src, T, R1, out, O2, n2, L, kk, (int)k3, k1);
        else
            rowx_go<SF, SOut, 32>(cx, rp, src, T, R1, out, O2, n2, L, kk, (int)k3, k1);
        cx.check_launch();
    }


    // The first strided pass (dimension 1, view [n1, I]) with partial row
    // totals Rp (kernels_fold.cuh).
    template <class SIn, class SOut>
    static void fold_pass(Ctx &cx, const SIn *src, SOut *dst, int64_t n1, int64_t I, int64_t k1, int64_t L,
                          L_ *Rp)
    {
        if constexpr (sizeof(L_) == 4 && sizeof(SOut) == 4) {
            int Lc = 128;
            while (Lc > 2 * k1 && Lc > 16 && cdiv(n1, Lc) * (I / 4) < cx.sms * 1024) Lc >>= 1;
            if (Lc > 32) Lc = 32;
            if (Lc > n1) Lc = (int)n1;
            const int nchunks = (int)cdiv(n1, Lc);
            const int64_t total = nchunks * (I / 4);
            cx.before(TAG_INC_FOLD, n1 * I);
            if (k1 <= 4)
                k_inc_strided4_rt<M, SIn, SOut, 4><<<(unsigned)cdiv(total, 128), 128, 0, cx.stream>>>(
                    src, dst, (int)n1, I, (int)k1, Lc, nchunks, (int)L, Rp);
            else
                k_inc_strided4_rt<M, SIn, SOut, 8><<<(unsigned)cdiv(total, 128), 128, 0, cx.stream>>>(
                    src, dst, (int)n1, I, (int)k1, Lc, nchunks, (int)L, Rp);
            cx.check_launch();
        }
    }

    // The two-dimensional lower problem T = excluded(R, (k1, k2)) of an
    // [n1, n2] tensor of row totals: plane totals R2 (from the H partials
    // of each row in P, writing R too, or from R itself with P == R, H == 1
    // and Rw null), then one block per plane (kernels_fold.cuh).
    template <class SP>
    static void lower2d(Ctx &cx, const SP *P, int H, CAR *Rw, const CAR *R, CAR *R2, CAR *T, int64_t n1,
                        int64_t n2, int64_t k1, int64_t k2, bool pdl = false)
    {
        if (cx.dry || !cx.ok()) return;
        cx.level++;
        cx.before(TAG_PLANE, n1 * n2);
        if (pdl)
            launch_pdl(k_plane_totals<MC, SP>, (unsigned)n1, 256, 0, cx.stream, P, H, Rw, R2, (int)n2);
        else
            k_plane_totals<MC, SP><<<(unsigned)n1, 256, 0, cx.stream>>>(P, H, Rw, R2, (int)n2);
        cx.check_launch();
        cx.before(TAG_EXC2D, n1 * n2);
        exc2d_launch<CAR, CAR>(cx, R, R2, T, n1, n2, k1, k2, pdl, 0);
        cx.level--;
    }

    // Excluded sums of the n1 x n2 array R with box (k1, k2) from its plane
    // totals R2 (r_ready: R is not written by the kernel before, so the block
    // kernel reads its window of planes before waiting for R2): one warp per plane (k_exc2d_w) when there are planes enough
    // to fill the GPU that way, else one block per plane (k_exc2d: a few
    // planes each get a whole block's parallelism).
    template <class SR, class ST>
    static void exc2d_launch(Ctx &cx, const SR *R, const CAR *R2, ST *T, int64_t n1, int64_t n2, int64_t k1,
                             int64_t k2, bool pdl, int r_ready)
    {
        using Acc = typename MC::acc_t;
        if (n1 < 8 * cx.sms) {
            const size_t smem = 2 * (size_t)n2 * sizeof(Acc);
            auto kern = k_exc2d<MC, SR, ST>;
            if (smem > 48 * 1024)
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (pdl)
                launch_pdl(kern, (unsigned)n1, 256, smem, cx.stream, R, R2, T, (int)n1, (int)n2, (int)k1, (int)k2,
                           r_ready);
            else
                kern<<<(unsigned)n1, 256, smem, cx.stream>>>(R, R2, T, (int)n1, (int)n2, (int)k1, (int)k2, r_ready);
            cx.check_launch();
            return;
        }
        const int wpb = exc2d_w_warps((int)n2, (int)sizeof(Acc));
        const size_t smem = 2 * (size_t)wpb * n2 * sizeof(Acc);
        auto kern = k_exc2d_w<MC, SR, ST>;
        if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const unsigned grid = (unsigned)cdiv(n1, wpb);
        if (pdl)
            launch_pdl(kern, grid, 32 * wpb, smem, cx.stream, R, R2, T, (int)n1, (int)n2, (int)k1, (int)k2);
        else
            kern<<<grid, 32 * wpb, smem, cx.stream>>>(R, R2, T, (int)n1, (int)n2, (int)k1, (int)k2);
        cx.check_launch();
    }

    template <class SIn, class SOut>
    static void excluded_rows(Ctx &cx, const RowPlan &rp, const SIn *X, SOut *out, int d,
                              const int64_t *n, const int64_t *k)
    {
        int64_t N = 1;
        for (int i = 0; i < d; ++i) N *= n[i];
        const int64_t L = n[d - 1], rows = N / L, n2 = n[d - 2], O2 = rows / n2;
        // BDBS passes before the final one: dimensions 1..d-2, and d-1 unless
        // the final pass takes its window.
        int dims[16];
        int P = 0;
        for (int j = 0; j < d - 2; ++j)
            if (k[j] > 1) dims[P++] = j;
        if (k[d - 2] > 1 && !rp.fuse) dims[P++] = d - 2;
        SOut *B = P > 0 ? cx.take<SOut>(N) : nullptr;
        SOut *B2 = P > 1 ? cx.take<SOut>(N) : nullptr;
        CAR *R = cx.take<CAR>(rows);
        CAR *T = cx.take<CAR>(rows);
        // d = 3: the lower problem is two-dimensional and, for boxes k1 <= 64
        // and planes of at most 4096 rows, takes two short kernels.  When the
        // first pass is the 16-byte strided pass along dimension 1 over rows
        // of whole 128-element groups, it also leaves partial row totals, and
        // X is read once instead of twice (kernels_fold.cuh).
        const bool lower2 = d == 3 && n[1] <= 4096 && k[0] <= 64 && n[0] <= SMALL2D_N1;
        bool fold = false;
        if constexpr (sizeof(L_) == 4 && sizeof(SOut) == 4)
            fold = lower2 && !rp.longrow && P > 0 && dims[0] == 0 && (L % 128) == 0 && k[0] <= 8 &&
                   env_int("EXSUM_FOLD", 1) != 0;
        CAR *R2 = lower2 ? cx.take<CAR>(n[0]) : nullptr;
        L_ *Rp = fold ? cx.take<L_>(rows * (L / 128)) : nullptr;
        if (fold && !cx.dry && cx.ok()) {
            SOut *dst0 = ((P - 1) % 2 == 0) ? B : B2;
            if ((((uintptr_t)X) & (sizeof(SIn) * 4 - 1)) || (((uintptr_t)dst0) & 15)) fold = false;
        }
        if (fold) {
            // everything on the caller's stream: pass 1 (+ partial row
            // totals) -> plane totals -> lower excluded sums -> final pass
            if (cx.dry || !cx.ok()) return;
            SOut *dst0 = ((P - 1) % 2 == 0) ? B : B2;
            int64_t I = N / n[0];
            // the kernels after the first are launched programmatically
            // dependent (each waits for the one before; launch latency hidden)
            const bool pdl = env_int("EXSUM_PDL", 1) != 0;
            fold_pass<SIn, SOut>(cx, X, dst0, n[0], I, k[0], L, Rp);
            lower2d<L_>(cx, Rp, (int)(L / 128), R, R, R2, T, n[0], n[1], k[0], k[1], pdl);
            const void *cur = dst0;
            for (int p = 1; p < P; ++p) {
                const int j = dims[p];
                int64_t O = 1;
                I = 1;
                for (int m = 0; m < j; ++m) O *= n[m];
                for (int m = j + 1; m < d; ++m) I *= n[m];
                SOut *dst = ((P - 1 - p) % 2 == 0) ? B : B2;
                inc_pass<SOut, SOut>(cx, (const SOut *)cur, dst, O, n[j], I, k[j]);
                cur = dst;
            }
            rowx_launch<SOut, SOut>(cx, rp, (const SOut *)cur, T, nullptr, out, O2, n2, L, k[d - 2], k[d - 1],
                                    pdl && P == 1);
            return;
        }
        // Row totals and the lower-dimensional recursion run on the side
        // stream while the BDBS passes run on the caller's.  A one-dimensional
        // recursion of at most ROWX_TAIL elements is left to the final pass
        // (it needs only R).
        const bool tail = !rp.longrow && d == 2 && n[0] <= ROWX_TAIL && k[0] <= 64;
        const Aux *aux = cx.aux;
        const bool fork = P > 0 && aux && aux->side && !cx.dry && cx.ok();
        cudaStream_t main_stream = cx.stream;
        if (fork) {
            cudaEventRecord(aux->fork, main_stream);
            cudaStreamWaitEvent(aux->side, aux->fork, 0);
            cx.stream = aux->side;
        }
        cx.aux = nullptr;
        if (!cx.dry && cx.ok()) {
            cx.before(TAG_ROWSUM, N);
            const int lpr = row_lanes(L);
            int64_t blocks = cdiv(rows, 8 * 4 * (32 / lpr));
            if (blocks > cx.sms * 8) blocks = cx.sms * 8;
            if (lpr <= 4)
                k_row_totals<M, SIn, 4><<<(unsigned)blocks, 256, 0, cx.stream>>>(X, R, rows, (int)L);
            else if (lpr == 8)
                k_row_totals<M, SIn, 8><<<(unsigned)blocks, 256, 0, cx.stream>>>(X, R, rows, (int)L);
            else if (lpr == 16)
                k_row_totals<M, SIn, 16><<<(unsigned)blocks, 256, 0, cx.stream>>>(X, R, rows, (int)L);
            else
                k_row_totals<M, SIn, 32><<<(unsigned)blocks, 256, 0, cx.stream>>>(X, R, rows, (int)L);
            cx.check_launch();
        }
        if (lower2) {
            lower2d<CAR>(cx, R, 1, nullptr, R, R2, T, n[0], n[1], k[0], k[1]);
        } else if (!tail) {
            cx.level++;
            Pipe<MC>::template excluded<CAR, CAR>(cx, R, T, d - 1, n, k);
            cx.level--;
        }
        cx.aux = aux;
        if (fork) {
            cudaEventRecord(aux->join, aux->side);
            cx.stream = main_stream;
        }
        const void *cur = X;
        for (int p = 0; p < P; ++p) {
            const int j = dims[p];
            int64_t O = 1, I = 1;
            for (int m = 0; m < j; ++m) O *= n[m];
            for (int m = j + 1; m < d; ++m) I *= n[m];
            SOut *dst = ((P - 1 - p) % 2 == 0) ? B : B2;
            if (p == 0)
                inc_pass<SIn, SOut>(cx, (const SIn *)cur, dst, O, n[j], I, k[j]);
            else
                inc_pass<SOut, SOut>(cx, (const SOut *)cur, dst, O, n[j], I, k[j]);
            cur = dst;
        }
        if (fork) cudaStreamWaitEvent(main_stream, aux->join, 0);
        const CAR *R1 = tail ? R : nullptr;
        if (P > 0)
            rowx_launch<SOut, SOut>(cx, rp, (const SOut *)cur, T, R1, out, O2, n2, L, k[d - 2], k[d - 1]);
        else
            rowx_launch<SIn, SOut>(cx, rp, (const SIn *)cur, T, R1, out, O2, n2, L, k[d - 2], k[d - 1]);
    }

    // ---- excluded sums: box-complement, one dimension-reduction step per level ---------------
    //
    // Level with input X of shape n[0..d-1]:
    //   H  = included sum of X along dimensions 2..d            (BDBS-Along-Dim)
    //   G  = total of X over dimension 1                          (dimension reduction)
    //   T  = excluded sum of G with box k[1..d-1]                 (next level)
    //   out[x] = prefix of H along dim 1 before x_1 (+) suffix of H along dim 1 from
    //            x_1+k_1 (+) T[x_2..x_d]
    // which is the two regions of step 1 in Corollary "Excluded-sum Components" plus
    // the regions of steps 2..d (all of which range over the whole of dimension 1).
    template <class SIn, class SOut>
    static void excluded(Ctx &cx, const SIn *X, SOut *out, int d, const int64_t *n,
                         const int64_t *k)
    {
        if (!cx.ok()) return;
        int64_t N = 1;
        for (int i = 0; i < d; ++i) N *= n[i];
        const int64_t M1 = N / n[0];
        if (d == 1) {
            exline_stage<SIn, SOut>(cx, X, nullptr, out, n[0], 1, k[0]);
            return;
        }
        // A small two-dimensional tensor: plane totals, then one block per
        // row of the output (kernels_fold.cuh), the whole sum in the long
        // accumulator -- two short kernels instead of a chain of passes.
        // (every plane combines all plane totals: n_1 is bounded so that
        // this stays far below the tensor's own cost)
        if (d == 2 && n[1] <= 4096 && n[0] <= SMALL2D_N1 && k[0] <= 64 && N <= (1 << 20) &&
            k[0] * N <= (1 << 24) && env_int("EXSUM_SMALL2D", 1) != 0) {
            CAR *R2 = cx.take<CAR>(n[0]);
            if (cx.dry || !cx.ok()) return;
            cx.before(TAG_PLANE, N);
            k_plane_totals<MC, SIn><<<(unsigned)n[0], 256, 0, cx.stream>>>(X, 1, nullptr, R2, (int)n[1]);
            cx.check_launch();
            cx.before(TAG_EXC2D, N);
            exc2d_launch<SIn, SOut>(cx, X, R2, out, n[0], n[1], k[0], k[1], true, 1);
            return;
        }
        RowPlan rp = row_plan(d, n, k, cx.sms);
        if (!rp.ok) rp = long_row_plan(d, n);
        if (rp.ok) {
            excluded_rows<SIn, SOut>(cx, rp, X, out, d, n, k);
            return;
        }
        const int64_t S = cdiv(n[0], EXL);
        int dims[16];
        int P = 0;
        for (int j = d - 1; j >= 1; --j)
            if (k[j] > 1) dims[P++] = j;
        // H ping-pongs between two workspace buffers and ends in B; `out` is
        // written once, by the last kernel, and never used as scratch.
        SOut *B = P > 0 ? cx.take<SOut>(N) : nullptr;
        SOut *B2 = P > 1 ? cx.take<SOut>(N) : nullptr;
        CAR *R = cx.take<CAR>(S * M1);
        CAR *Rt = cx.take<CAR>(S * M1);
        CAR *G = cx.take<CAR>(M1);
        CAR *T = cx.take<CAR>(M1);
        CAR *Qa = S > 1 ? cx.take<CAR>(S * M1) : nullptr;
        const bool blk = S > 64 && M1 < 4096;
        CAR *SR = (S > 1 && blk) ? cx.take<CAR>(S * M1) : nullptr;
        const int r_tail = (int)(k[0] % EXL);
        // The first pass fuses the segment totals of X when it is the
        // contiguous register pass over whole 32-row segments.
        const bool fused = P > 0 && dims[0] == d - 1 && k[d - 1] <= 32 && n[0] >= 32;
        // H: BDBS along dims d..2, ending in B.  Pass 0 runs first; when it carries the segment totals, the carries,
        // their included sums and the lower-dimensional recursion only depend
        // on it and run on the side stream while the other passes proceed.
        auto run_pass = [&](int p, const void *src) -> SOut * {
            const int j = dims[p];
            int64_t O = 1, I = 1;
            for (int m = 0; m < j; ++m) O *= n[m];
            for (int m = j + 1; m < d; ++m) I *= n[m];
            SOut *dst = ((P - 1 - p) % 2 == 0) ? B : B2;
            if (p == 0 && fused) {
                if (!cx.dry && cx.ok()) {
                    const int64_t kk = k[j];
                    if (kk <= 4)
                        inc_fast<SIn, SOut, 4>(cx, (const SIn *)src, dst, O, n[j], I, kk, n[0], R, Rt, r_tail);
                    else if (kk <= 8)
                        inc_fast<SIn, SOut, 8>(cx, (const SIn *)src, dst, O, n[j], I, kk, n[0], R, Rt, r_tail);
                    else if (kk <= 16)
                        inc_fast<SIn, SOut, 16>(cx, (const SIn *)src, dst, O, n[j], I, kk, n[0], R, Rt, r_tail);
                    else
                        inc_fast<SIn, SOut, 32>(cx, (const SIn *)src, dst, O, n[j], I, kk, n[0], R, Rt, r_tail);
                }
            } else if (p == 0) {
                inc_pass<SIn, SOut>(cx, (const SIn *)src, dst, O, n[j], I, k[j]);
            } else {
                inc_pass<SOut, SOut>(cx, (const SOut *)src, dst, O, n[j], I, k[j]);
            }
            return dst;
        };
        const void *cur = X;
        int p_next = 0;
        if (fused) cur = run_pass(p_next++, cur);
        // Fork.
        const Aux *aux = cx.aux;
        const bool fork = aux && aux->side && !cx.dry && cx.ok();
        cudaStream_t main_stream = cx.stream;
        if (fork) {
            cudaEventRecord(aux->fork, main_stream);
            cudaStreamWaitEvent(aux->side, aux->fork, 0);
            cx.stream = aux->side;
        }
        cx.aux = nullptr;
        if (!fused && !cx.dry && cx.ok()) {
            cx.before(TAG_REDUCE, N);
            k_reduce_seg2<M, SIn><<<(unsigned)cdiv(S * M1, 256), 256, 0, cx.stream>>>(
                X, R, Rt, n[0], M1, EXL, S, r_tail);
            cx.check_launch();
        }
        // Carries of the dimension-1 step and the column totals G.
        if (!cx.dry && cx.ok()) {
            const int64_t qoff = 1 + k[0] / EXL;
            cx.before(TAG_CARRY, S * M1);
            if (S > 1 && blk)
                k_carry_blk<M, 1024><<<(unsigned)M1, 1024, 0, cx.stream>>>(R, Rt, nullptr, Qa, SR,
                                                                           M1, S, qoff, G);
            else
                k_carry_qa<M><<<(unsigned)cdiv(M1, 256), 256, 0, cx.stream>>>(R, Rt, Qa, G, M1, S,
                                                                              qoff);
            cx.check_launch();
        }
        // Second branch: the lower-dimensional recursion only needs G; it runs
        // on side2 while the carries' included sums run on side.
        const bool fork2 = fork && aux->side2;
        if (fork2) {
            cudaEventRecord(aux->fork2, cx.stream);
            cudaStreamWaitEvent(aux->side2, aux->fork2, 0);
        }
        // Included sums of the carries along dims 2..d (view [S, n_2, .., n_d]).
        CAR *Qh = Qa;
        if (S > 1 && P > 0) {
            int64_t ns[16], ks[16];
            ns[0] = S;
            ks[0] = 1;
            for (int m = 1; m < d; ++m) {
                ns[m] = n[m];
                ks[m] = k[m];
            }
            CAR *Qo = cx.take<CAR>(S * M1);
            Pipe<MC>::template included<CAR, CAR>(cx, Qa, Qo, d, ns, ks);
            Qh = Qo;
        }
        if (fork2) cx.stream = aux->side2;
        cx.level++;
        Pipe<MC>::template excluded<CAR, CAR>(cx, G, T, d - 1, n + 1, k + 1);
        cx.level--;
        // Join: the remaining passes on the caller's stream, then wait.
        cx.aux = aux;
        if (fork) {
            cudaEventRecord(aux->join, aux->side);
            if (fork2) cudaEventRecord(aux->join2, aux->side2);
            cx.stream = main_stream;
        }
        for (; p_next < P; ++p_next) cur = run_pass(p_next, cur);
        if (fork) cudaStreamWaitEvent(main_stream, aux->join, 0);
        if (fork2) cudaStreamWaitEvent(main_stream, aux->join2, 0);
        if (!cx.dry && cx.ok()) {
            cx.before(TAG_EXLINE, N);
            if (P > 0)
                exline_launch<SOut, SOut>(cx, B, Qh, T, out, n[0], M1, k[0], S);
            else
                exline_launch<SIn, SOut>(cx, X, Qh, T, out, n[0], M1, k[0], S);
            cx.check_launch();
        }
    }

    // ---- entry -----------------------------------------------------------------------------
    static int run(int excluded_sum, const void *in, void *out, int d, const int64_t *n,
                   const int64_t *k, void *ws, size_t ws_bytes, cudaStream_t stream,
                   size_t *ws_needed, cudaError_t *cuda_err, const Aux *aux)
    {
        Ctx cx;
        cx.dry = true;
        cx.sms = device_sms();
        if (excluded_sum)
            excluded<IN, OUT>(cx, nullptr, nullptr, d, n, k);
        else
            included<IN, OUT>(cx, nullptr, nullptr, d, n, k);
        const size_t need = cx.off;
        if (ws_needed) *ws_needed = need;
        if (!in) return ST_OK;  // size query only
        if (need > ws_bytes || (need > 0 && !ws)) return ST_ENOMEM;
        Ctx rx;
        rx.dry = false;
        rx.sms = cx.sms;
        rx.base = (char *)ws;
        rx.cap = ws_bytes;
        rx.stream = stream;
        rx.aux = aux;
        if (excluded_sum)
            excluded<IN, OUT>(rx, (const IN *)in, (OUT *)out, d, n, k);
        else
            included<IN, OUT>(rx, (const IN *)in, (OUT *)out, d, n, k);
        if (cuda_err) *cuda_err = rx.cuda_err;
        return rx.status;
    }
};

}  // namespace exsum
