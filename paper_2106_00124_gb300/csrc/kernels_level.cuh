// kernels_level.cuh -- multi-tensor kernels: one launch runs one pass level
// of the row schedule (Sec. 4) for every tensor of a batch.
//
// A batch of excluded sums is a set of independent pass chains (strided BDBS
// pass, row totals, plane totals, the two-dimensional lower problem, the
// final pass).  Instead of one launch per pass per tensor, the planner
// (exsum_level.cu) writes, for each level, a work list of items -- an item is
// a run of consecutive virtual blocks of one pass of one tensor, with that
// pass's parameters and the index of its first virtual block -- and a table
// giving the item of every work-list slot.  A level is one launch (per
// register class): block b runs slot b, the hardware block scheduler handing
// out the slots as blocks finish; or, as a tuning option, a persistent grid
// of a few blocks per SM pulls slots from a device counter.  The pass bodies
// are the single-tensor kernels' own (`*_body`), called with a virtual
// block index and grid, so a tensor's results do not depend on which
// physical block computed which part, nor on the order of the slots.
#pragma once

#include "kernels_fold.cuh"
#include "kernels_rowbulk.cuh"

namespace exsum {

// Body selectors.  Level 1 (128 threads): BDBS along a strided dimension
// (4 inner positions per thread or 1) and row totals; plane totals and the
// lower problem (256 threads); the final pass (256 threads): staged by bulk
// copies or by k_rowx's 16-byte asynchronous copies.
enum LvKind : int {
    LV_S4_K4 = 0, LV_S4_K8, LV_S1_K4, LV_S1_K8, LV_S1_K16, LV_S1_K32,
    LV_RT_4, LV_RT_8, LV_RT_16, LV_RT_32,
    LV_PT_IN, LV_PT_CAR,                 // plane totals of the input (d = 2) / of R (d = 3)
    LV_E2_IN, LV_E2_CAR,                 // lower problem of the input (d = 2) / of R (d = 3)
    LV_BK_K1, LV_BK_K8, LV_BK_K32,       // bulk-staged final pass, window bound 1, 8, 32
    LV_RX_K1_E4, LV_RX_K1_E8, LV_RX_K1_E16, LV_RX_K1_E32,
    LV_RX_K8_E4, LV_RX_K8_E8, LV_RX_K8_E16, LV_RX_K8_E32,
    LV_RX_K32_E4, LV_RX_K32_E8, LV_RX_K32_E16, LV_RX_K32_E32,
    // window sums along x1 of the lower problem's input (H1), from the carry
    // type (d = 3: R) or the input type (d = 2: X), window bound 4 .. 32
    LV_H1C_K4, LV_H1C_K8, LV_H1C_K16, LV_H1C_K32,
    LV_H1I_K4, LV_H1I_K8, LV_H1I_K16, LV_H1I_K32,
    LV_E2_CO,                            // lower problem from H1 (carry type) into the output (d = 2)
    LV_KINDS
};

// One work-list item.  Slots [off, off + count) of the level map to the
// pass's virtual blocks [vbase, vbase + count) of a virtual grid of vgrid.
struct LvItem {
    int64_t off, count, vbase, vgrid;
    const void *src;   // pass input
    void *dst;         // pass output
    const void *t;     // final pass: T; lower problem: R2
    void *r;           // row totals: R; plane totals: R2
    int64_t O, I;      // strided view [O, n, I]; row totals: rows; final pass: slices
    int kind;
    int n, k, Lc, nchunks;                                   // strided pass
    int L, n2, k2, k3, TR, GO, ntile, RS, RSA, LS, lpr;      // final pass, lower problem
    int aligned, LSW, ntiles;                                // bulk final pass
    int pad_;
};

// A level's work list: the items, the item of every slot, the slot count
// and, for a persistent grid, the counter its blocks pull slots from (null:
// one block per slot, handed out by the hardware's block scheduler).
struct LvList {
    const LvItem *items;
    const int *slot_item;
    int64_t nslots;
    unsigned long long *ctr;
};

// Runs the level's slots: `run(item, virtual block)` returns false to stop
// the block (a bounded wait that gave up).  Without PERSIST a block runs the
// one slot of its index (the hardware's block scheduler hands the slots
// out as blocks finish); with PERSIST a grid of a few blocks per SM pulls
// slots from the list's counter, each block pulling its next slot while it
// runs the current one.  (The loop costs registers: in this form the bodies
// spill, so it is a tuning choice, not the default.)
template <bool PERSIST, class F>
__device__ __forceinline__ void lv_pull(const LvList &ls, F run)
{
    if constexpr (!PERSIST) {
        const int64_t slot = blockIdx.x;
        const LvItem &w = ls.items[ls.slot_item[slot]];
        run(w, w.vbase + (slot - w.off));
    } else {
        __shared__ long long s_slot[2];
        if (threadIdx.x == 0) s_slot[0] = (long long)atomicAdd(ls.ctr, 1ull);
        int buf = 0;
        for (;;) {
            __syncthreads();   // s_slot[buf] is written; the previous body is done with shared memory
            const int64_t slot = s_slot[buf];
            if (slot >= ls.nslots) return;
            long long next = 0;
            if (threadIdx.x == 0) next = (long long)atomicAdd(ls.ctr, 1ull);
            const LvItem &w = ls.items[ls.slot_item[slot]];
            if (!run(w, w.vbase + (slot - w.off))) return;
            if (threadIdx.x == 0) s_slot[buf ^ 1] = next;
            buf ^= 1;
        }
    }
}

// Register classes: a level kernel is compiled for the largest body it
// runs, so bodies of very different register needs go to separate kernels
// (each keeps about the occupancy its bodies have as single-tensor
// kernels).  Level 1: class 0 at most 64 registers, class 1 at most 80.
// Final pass (k_rowx): class 0 at most 64, class 1 at most 128, class 2
// (strips of 32 elements) up to 255.
__host__ __device__ constexpr int lv_class(int kind)
{
    if (kind == LV_S1_K32 || kind == LV_S4_K8) return 1;
    if (kind == LV_H1C_K32 || kind == LV_H1I_K32) return 1;
    if (kind >= LV_RX_K1_E4 && kind <= LV_RX_K32_E32) {
        const int km = (kind - LV_RX_K1_E4) / 4, e = (kind - LV_RX_K1_E4) % 4;   // km 0: 1, 1: 8, 2: 32
        if (e == 3) return 2;
        return (km < 2 && e < 2) ? 0 : 1;
    }
    return 0;
}

// The bodies, with their parameters taken from a work-list item.
template <class M, int KMAX, bool V4>
__device__ __forceinline__ void lv_strided(const LvItem &w, int64_t vb)
{
    using Lt = typename M::loc_t;
    const Lt *src = static_cast<const Lt *>(w.src);
    Lt *dst = static_cast<Lt *>(w.dst);
    if constexpr (V4)
        k_inc_strided4_body<M, Lt, Lt, KMAX>(src, dst, w.O, w.n, w.I, w.k, w.Lc, w.nchunks, vb, w.vgrid);
    else
        k_inc_strided_body<M, Lt, Lt, KMAX>(src, dst, w.O, w.n, w.I, w.k, w.Lc, w.nchunks, vb, w.vgrid);
}

template <class M, int LPR>
__device__ __forceinline__ void lv_rowtot(const LvItem &w, int64_t vb)
{
    using Lt = typename M::loc_t;
    k_row_totals_body<M, Lt, LPR>(static_cast<const Lt *>(w.src), static_cast<typename M::car_t *>(w.r), w.O, w.L,
                                  vb, w.vgrid);
}

// ---- level 1: strided BDBS passes and row totals (128 threads) -------------------
template <class M, int CLS, bool PERSIST>
__global__ void __launch_bounds__(128, CLS == 0 ? 8 : 6)
kl_stage1(LvList ls)
{
    // the second strided pass reads the first's output: the input must be
    // the local type
    static_assert(std::is_same<typename M::in_t, typename M::loc_t>::value, "input read as the local type");
    lv_pull<PERSIST>(ls, [&](const LvItem &w, int64_t vb) {
        if constexpr (CLS == 0) {
            switch (w.kind) {
            case LV_S4_K4: lv_strided<M, 4, true>(w, vb); break;
            case LV_S1_K4: lv_strided<M, 4, false>(w, vb); break;
            case LV_S1_K8: lv_strided<M, 8, false>(w, vb); break;
            case LV_S1_K16: lv_strided<M, 16, false>(w, vb); break;
            case LV_RT_4: lv_rowtot<M, 4>(w, vb); break;
            case LV_RT_8: lv_rowtot<M, 8>(w, vb); break;
            case LV_RT_16: lv_rowtot<M, 16>(w, vb); break;
            case LV_RT_32: lv_rowtot<M, 32>(w, vb); break;
            default: break;
            }
        } else {
            if (w.kind == LV_S4_K8)
                lv_strided<M, 8, true>(w, vb);
            else
                lv_strided<M, 32, false>(w, vb);
        }
        return true;
    });
}

// ---- plane totals (256 threads): one virtual block per plane x1 -----------------
// M is the monoid of the carries (compensated arithmetic for fp +).
template <class M, bool PERSIST>
__global__ void __launch_bounds__(256)
kl_plane(LvList ls)
{
    using IN = typename M::in_t;
    using C = typename M::car_t;
    lv_pull<PERSIST>(ls, [&](const LvItem &w, int64_t vb) {
        C *R2 = static_cast<C *>(w.r);
        if (w.kind == LV_PT_IN)
            k_plane_totals_body<M, IN>(static_cast<const IN *>(w.src), 1, nullptr, R2, w.n2, vb, w.vgrid);
        else
            k_plane_totals_body<M, C>(static_cast<const C *>(w.src), 1, nullptr, R2, w.n2, vb, w.vgrid);
        return true;
    });
}

// ---- window sums along x1 of the lower problem (128 threads) ---------------------
// M is the monoid of the carries; the strided BDBS pass over the view
// [1, n1, n2] of R (or X), into H1 in the carry type.
template <class M, int CLS, bool PERSIST>
__global__ void __launch_bounds__(128, CLS == 0 ? 6 : 3)
kl_lower_h1(LvList ls)
{
    using IN = typename M::in_t;
    using C = typename M::car_t;
    lv_pull<PERSIST>(ls, [&](const LvItem &w, int64_t vb) {
        C *dst = static_cast<C *>(w.dst);
        const C *sc = static_cast<const C *>(w.src);
        const IN *si = static_cast<const IN *>(w.src);
        auto hc = [&](auto kk) {
            k_inc_strided_body<M, C, C, decltype(kk)::value>(sc, dst, w.O, w.n, w.I, w.k, w.Lc, w.nchunks, vb,
                                                             w.vgrid);
        };
        auto hi = [&](auto kk) {
            k_inc_strided_body<M, IN, C, decltype(kk)::value>(si, dst, w.O, w.n, w.I, w.k, w.Lc, w.nchunks, vb,
                                                              w.vgrid);
        };
        if constexpr (CLS == 0) {
            switch (w.kind) {
            case LV_H1C_K4: hc(std::integral_constant<int, 4>()); break;
            case LV_H1C_K8: hc(std::integral_constant<int, 8>()); break;
            case LV_H1C_K16: hc(std::integral_constant<int, 16>()); break;
            case LV_H1I_K4: hi(std::integral_constant<int, 4>()); break;
            case LV_H1I_K8: hi(std::integral_constant<int, 8>()); break;
            default: hi(std::integral_constant<int, 16>()); break;
            }
        } else {
            if (w.kind == LV_H1C_K32)
                hc(std::integral_constant<int, 32>());
            else
                hi(std::integral_constant<int, 32>());
        }
        return true;
    });
}

// ---- the two-dimensional lower problem (128 threads): one warp per x1 ----------
// d = 3: T = excluded(R) in the carry type; d = 2: the output itself.
template <class M, bool PERSIST>
__global__ void __launch_bounds__(128)
kl_exc2d(LvList ls)
{
    using IN = typename M::in_t;
    using OUT = typename M::out_t;
    using C = typename M::car_t;
    lv_pull<PERSIST>(ls, [&](const LvItem &w, int64_t vb) {
        const C *R2 = static_cast<const C *>(w.t);
        const int kwin = w.Lc > 0 ? w.Lc : w.k;   // Lc: planes per window read here (1: H1 given)
        if (w.kind == LV_E2_IN)
            k_exc2d_w_body<M, IN, OUT>(static_cast<const IN *>(w.src), R2, static_cast<OUT *>(w.dst), w.n, w.n2,
                                       w.k, w.k2, vb, w.vgrid, kwin);
        else if (w.kind == LV_E2_CO)
            k_exc2d_w_body<M, C, OUT>(static_cast<const C *>(w.src), R2, static_cast<OUT *>(w.dst), w.n, w.n2,
                                      w.k, w.k2, vb, w.vgrid, kwin);
        else
            k_exc2d_w_body<M, C, C>(static_cast<const C *>(w.src), R2, static_cast<C *>(w.dst), w.n, w.n2, w.k,
                                    w.k2, vb, w.vgrid, kwin);
        return true;
    });
}

// ---- final pass, staged by bulk copies (256 threads, two blocks per SM) ----------
template <class M, int KMAX, bool ODD>
__device__ __forceinline__ bool lv_bulk(const LvItem &w, int64_t vb)
{
    using Lt = typename M::loc_t;
    using OUT = typename M::out_t;
    return k_rowx_bulk_body<M, OUT, KMAX, 32, 2, 256, 0, ODD>(
        static_cast<const Lt *>(w.src), static_cast<const typename M::car_t *>(w.t), static_cast<OUT *>(w.dst),
        w.ntiles, w.ntile, w.n2, w.L, w.k2, w.k3, w.TR, w.LSW, w.lpr, w.aligned, vb, w.vgrid);
}

// ODD: rows whose length is not a multiple of 4 (a launch of their own)
template <class M, bool PERSIST, bool ODD>
__global__ void __launch_bounds__(256, 2)
kl_final_bulk(LvList ls)
{
    lv_pull<PERSIST>(ls, [&](const LvItem &w, int64_t vb) -> bool {
        switch (w.kind) {
        case LV_BK_K1: return lv_bulk<M, 1, ODD>(w, vb);
        case LV_BK_K8: return lv_bulk<M, 8, ODD>(w, vb);
        default: return lv_bulk<M, 32, ODD>(w, vb);
        }
    });
}

// ---- final pass, k_rowx (256 threads): one virtual block per tile -----------------
template <class M, int KM, int EPL>
__device__ __forceinline__ void lv_rowx(const LvItem &w, int64_t vb)
{
    using Lt = typename M::loc_t;
    using OUT = typename M::out_t;
    k_rowx_body<M, Lt, OUT, KM, EPL>(static_cast<const Lt *>(w.src), static_cast<const typename M::car_t *>(w.t),
                                     nullptr, 0, static_cast<OUT *>(w.dst), w.O, w.n2, w.L, w.k2, w.k3, w.TR, w.GO,
                                     w.ntile, w.RS, w.RSA, w.LS, w.lpr, vb, w.vgrid);
}

template <class M, int CLS, bool PERSIST>
__global__ void __launch_bounds__(256, CLS == 0 ? 4 : CLS == 1 ? 2 : 1)
kl_final_rowx(LvList ls)
{
    lv_pull<PERSIST>(ls, [&](const LvItem &w, int64_t vb) {
        if constexpr (CLS == 0) {
            switch (w.kind) {
            case LV_RX_K1_E4: lv_rowx<M, 1, 4>(w, vb); break;
            case LV_RX_K1_E8: lv_rowx<M, 1, 8>(w, vb); break;
            case LV_RX_K8_E4: lv_rowx<M, 8, 4>(w, vb); break;
            default: lv_rowx<M, 8, 8>(w, vb); break;
            }
        } else if constexpr (CLS == 1) {
            switch (w.kind) {
            case LV_RX_K1_E16: lv_rowx<M, 1, 16>(w, vb); break;
            case LV_RX_K8_E16: lv_rowx<M, 8, 16>(w, vb); break;
            case LV_RX_K32_E4: lv_rowx<M, 32, 4>(w, vb); break;
            case LV_RX_K32_E8: lv_rowx<M, 32, 8>(w, vb); break;
            default: lv_rowx<M, 32, 16>(w, vb); break;
            }
        } else {
            switch (w.kind) {
            case LV_RX_K1_E32: lv_rowx<M, 1, 32>(w, vb); break;
            case LV_RX_K8_E32: lv_rowx<M, 8, 32>(w, vb); break;
            default: lv_rowx<M, 32, 32>(w, vb); break;
            }
        }
        return true;
    });
}

}  // namespace exsum
