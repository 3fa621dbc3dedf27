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
#include <string.h>

#include <type_traits>

#include "kernels_flat.cuh"

namespace exsum {

// Status codes, mirrored from include/exsum.h (kept numerically identical).
enum { ST_OK = 0, ST_EINVAL = -1, ST_ENOMEM = -2, ST_EUNSUP = -3, ST_ECUDA = -4 };

// Kernel tags reported by the launch trace (exsum_trace_*).
enum KernelTag {
    TAG_INC = 0,          // BDBS-Along-Dim, generic line pass (k > 32)
    TAG_REDUCE = 1,       // segment / column reductions
    TAG_SUMSEG = 2,       // segment totals -> column totals
    TAG_CARRY = 3,        // dimension-1 carries
    TAG_EXLINE = 4,       // dimension-1 prefix/suffix + contributions
    TAG_INC_CONTIG = 5,   // BDBS-Along-Dim, contiguous dimension (k_inc_flat)
    TAG_INC_STRIDED = 6,  // BDBS-Along-Dim, strided dimension (k_inc_strided)
    TAG_COUNT = 7
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

template <class M>
struct Pipe {
    // Monoid for work on carries (compensated local arithmetic for fp +).
    using MC = typename std::conditional<M::compensated, MonComp<M>, M>::type;
    using A = typename M::acc_t;
    using IN = typename M::in_t;
    using OUT = typename M::out_t;
    using CAR = typename M::car_t;

    static constexpr int EXL = 32;            // segment length of the dimension-1 step
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
            // Chunks short enough for ~2048 threads per SM (walks of a few blocks).
            int Lc = 128;
            while (Lc > 2 * k && Lc > 16 && O * cdiv(n, Lc) * I < 152 * 2048) Lc >>= 1;
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
        // Large boxes: per-thread suffix slots in shared or global memory.
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

    // ---- column totals over dimension 1 of a view [n1, Mc] ----------------------------
    template <class SIn>
    static void colsum(Ctx &cx, const SIn *X, CAR *G, int64_t n1, int64_t Mc)
    {
        if (!cx.ok()) return;
        int64_t S = cdiv(152 * 2048, Mc);
        if (S > cdiv(n1, 8)) S = cdiv(n1, 8);
        if (S < 1) S = 1;
        const int64_t L = cdiv(n1, S);
        S = cdiv(n1, L);
        if (S == 1) {
            if (cx.dry) return;
            cx.before(TAG_REDUCE, n1 * Mc);
            k_reduce_seg2<M, SIn><<<(unsigned)cdiv(Mc, 256), 256, 0, cx.stream>>>(X, G, nullptr, n1,
                                                                                   Mc, L, 1, 0);
            cx.check_launch();
            return;
        }
        CAR *Rx = cx.take<CAR>(S * Mc);
        if (cx.dry || !cx.ok()) return;
        cx.before(TAG_REDUCE, n1 * Mc);
        k_reduce_seg2<M, SIn><<<(unsigned)cdiv(S * Mc, 256), 256, 0, cx.stream>>>(X, Rx, nullptr, n1,
                                                                                   Mc, L, S, 0);
        cx.check_launch();
        cx.before(TAG_SUMSEG, S * Mc);
        if (Mc >= 1024)
            k_sum_segs_col<M><<<(unsigned)cdiv(Mc, 256), 256, 0, cx.stream>>>(Rx, G, Mc, S);
        else
            k_sum_segs_blk<M, 256><<<(unsigned)Mc, 256, 0, cx.stream>>>(Rx, G, Mc, S);
        cx.check_launch();
    }

    // ---- dimension-1 step: prefix/suffix along dim 1 + contributions --------------------
    static constexpr int CT_NT = 256, CT_V = 16, CT_L = CT_NT * CT_V;  // contiguous segment

    template <class SH, class SOut>
    static void exline_stage(Ctx &cx, const SH *H, const CAR *T, SOut *out, int64_t n1,
                             int64_t Mc, int64_t k1)
    {
        if (!cx.ok()) return;
        const bool contig = (Mc == 1);
        const int64_t L = contig ? CT_L : EXL;
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
            cx.before(TAG_REDUCE, n1 * Mc);
            if (contig)
                k_reduce_seg_contig<M, SH, CT_NT, CT_V><<<(unsigned)S, CT_NT, 0, cx.stream>>>(
                    H, R, Rt, n1, k1 % L);
            else
                k_reduce_seg2<M, SH><<<(unsigned)cdiv(S * Mc, 256), 256, 0, cx.stream>>>(
                    H, R, Rt, n1, Mc, L, S, k1 % L);
            cx.check_launch();
            const int64_t qoff = 1 + k1 / L;
            cx.before(TAG_CARRY, S * Mc);
            if (blk)
                k_carry_blk<M, 1024><<<(unsigned)Mc, 1024, 0, cx.stream>>>(R, Rt, T, Qb, SR, Mc, S,
                                                                           qoff, nullptr);
            else
                k_carry_col<M><<<(unsigned)cdiv(Mc, 256), 256, 0, cx.stream>>>(R, Rt, T, Qb, Mc, S,
                                                                                qoff);
            cx.check_launch();
            Q = Qb;
            qs = Mc;
        }
        if (cx.dry || !cx.ok()) return;
        cx.before(TAG_EXLINE, n1 * Mc);
        if (contig)
            k_exline_contig<M, SH, SOut, CT_NT, CT_V><<<(unsigned)S, CT_NT, 0, cx.stream>>>(
                H, Q, out, n1, k1);
        else
            k_exline2<M, SH, SOut, EXL><<<(unsigned)cdiv(S * Mc, 128), 128, 0, cx.stream>>>(
                H, Q, qs, nullptr, out, n1, Mc, k1, S);
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
