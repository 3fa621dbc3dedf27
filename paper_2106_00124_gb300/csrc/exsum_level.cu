// exsum_level.cu -- the level-batched schedule of a batch of excluded sums:
// every tensor's passes of one level run in one launch per register class
// over a device work list (kernels_level.cuh), so a batch of hundreds of
// tensors takes at most thirteen kernel launches (and, for persistent grids,
// one memset), whatever its size.
//
// A tensor joins a level set when its excluded sum takes the row schedule
// with the two-dimensional lower problem (d = 3, Sec. 4; n_2 <= 1024,
// n_1 <= 16384, rows of 16 .. 1024 elements, boxes of at most 32 along the
// strided passes) or the two short kernels of a small d = 2 tensor, and
// its operator and type are fp32 + (the type the level kernels are built
// for).  Its passes are those of the single-tensor path with the same
// tile plans (the lower problem excepted, see level 2), so the arithmetic is
// the same up to the order of the lower problem's window sums; only the work
// lists differ:
//   level 1   strided BDBS pass along dimension 1 (X -> B) and the row
//             totals R of X (d = 3);
//   level 1b  strided pass along dimension 2 (B2 -> B) when the final pass
//             does not take that window (side branch, beside levels 2, 3);
//   level 2   plane totals R2 (of R for d = 3, of X for d = 2), beside the
//             window sums H1 of R (or X) along dimension 1 by a strided
//             BDBS pass in the carry type;
//   level 3   the lower problem from H1 and R2, one warp per plane:
//             T = excluded(R) for d = 3, the output itself for d = 2;
//   level 4   the final pass (bulk-staged, or k_rowx on side branches).
// Each level's items are ordered largest tensor first, so the small ones
// fill the tail of the launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "kernels_level.cuh"
#include "level.h"
#include "pipeline.cuh"

namespace exsum {

namespace {

// levels; the strided and k_rowx levels in two register classes each
enum { LV1 = 0, LV1_C1, LV1B, LV1B_C1, LV2, LV2H, LV2H_C1, LV3, LV4A, LV4A_ODD, LV4B, LV4B_C1, LV4B_C2, NLV };

using M = M_F32_ADD;
using PM = Pipe<M>;
using MC = PM::MC;
using Lt = M::loc_t;
using C = M::car_t;
using AccC = MC::acc_t;

constexpr int kThreads[NLV] = {128, 128, 128, 128, 256, 128, 128, 128, 256, 256, 256, 256, 256};
// the lower problem: one warp per plane, four per block, each holding 2 n_2
// accumulators in shared memory (at most 64 KB a block)
constexpr int LV_E2_N2 = 1024;

int64_t cdiv64(int64_t a, int64_t b) { return (a + b - 1) / b; }

bool al16(const void *p) { return (((uintptr_t)p) & 15) == 0; }

}  // namespace

struct LevelSet {
    std::vector<LvItem> items[NLV];
    int64_t nslots[NLV] = {};
    size_t smem[NLV] = {};
    int grid[NLV] = {};
    LvItem *d_items = nullptr;
    int *d_slots = nullptr;              // item of every slot, all levels
    size_t slot_base[NLV] = {};
    bool persist = false;
    unsigned long long *d_ctr = nullptr;
    size_t item_base[NLV] = {};
    void *ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t side = nullptr;
    cudaStream_t side2 = nullptr;
    cudaEvent_t ev[6] = {};
    int sms = 152;
};

int level_sms() { return (int)device_sms(); }

bool level_accepts(const exsum_desc &d, int sms)
{
    if (d.op != EXSUM_OP_ADD || d.dtype != EXSUM_F32 || !d.in || !d.out) return false;
    int64_t N = 1;
    for (int i = 0; i < d.d; ++i) {
        if (d.shape[i] < 1 || d.k[i] < 1) return false;
        N *= d.shape[i];
    }
    const int64_t *n = d.shape, *k = d.k;
    if (d.d == 2) {
        // the small two-dimensional path of the single-tensor schedule
        return n[1] <= LV_E2_N2 && n[0] <= PM::SMALL2D_N1 && k[0] <= 32 && N <= (1 << 20) &&
               k[0] * N <= (1 << 24);
    }
    if (d.d != 3) return false;
    if (n[1] > LV_E2_N2 || k[0] > 32 || n[0] > PM::SMALL2D_N1 || N >= (1ll << 40)) return false;
    const auto rp = PM::row_plan(3, n, k, sms);
    if (!rp.ok) return false;
    if (!rp.fuse && k[1] > 32) return false;
    return true;
}

namespace {

// Workspace carving, identical in the sizing run (base null) and the real one.
struct Carver {
    char *base = nullptr;
    size_t off = 0;
    template <class T>
    T *take(int64_t n)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += (size_t)n * sizeof(T);
        return p;
    }
};

// A strided BDBS pass along the middle dimension of the view [O, n, I]:
// the body, its chunk length and its virtual grid (threads of 128).
struct StridedPlan {
    int kind = 0, Lc = 0, nchunks = 0;
    int64_t per_chunk = 0;   // threads per chunk (O == 1)
    int64_t vgrid = 0;
};

StridedPlan strided_plan(const void *src, const void *dst, int64_t O, int64_t n, int64_t I, int64_t k, int lc,
                         int sms)
{
    StridedPlan sp;
    const bool vec = k <= 8 && (I & 3) == 0 && al16(src) && al16(dst);
    const int64_t Iq = vec ? I / 4 : I;
    int Lc = 128;
    if (lc > 0) {
        Lc = lc;
    } else {
        // as the single-tensor pass: chunks short enough to give every SM
        // about 1024 (vector) or 2048 (scalar) threads, walks of a few blocks
        const int64_t want = (int64_t)sms * (vec ? 1024 : 2048);
        while (Lc > 2 * k && Lc > 16 && O * cdiv64(n, Lc) * Iq < want) Lc >>= 1;
    }
    if (Lc > n) Lc = (int)n;
    sp.Lc = Lc;
    sp.nchunks = (int)cdiv64(n, Lc);
    sp.per_chunk = Iq;
    sp.vgrid = cdiv64(O * sp.nchunks * Iq, 128);
    if (vec)
        sp.kind = k <= 4 ? LV_S4_K4 : LV_S4_K8;
    else
        sp.kind = k <= 4 ? LV_S1_K4 : k <= 8 ? LV_S1_K8 : k <= 16 ? LV_S1_K16 : LV_S1_K32;
    return sp;
}

LvItem strided_item(const StridedPlan &sp, const void *src, void *dst, int64_t O, int64_t n, int64_t I, int64_t k,
                    int64_t v0, int64_t v1)
{
    LvItem w{};
    w.kind = sp.kind;
    w.src = src;
    w.dst = dst;
    w.O = O;
    w.n = (int)n;
    w.I = I;
    w.k = (int)k;
    w.Lc = sp.Lc;
    w.nchunks = sp.nchunks;
    w.vgrid = sp.vgrid;
    w.vbase = v0;
    w.count = v1 - v0;
    return w;
}

// Row totals of `rows` rows of L elements: a piece of virtual blocks of 4
// warps, each block about 16K elements.
LvItem rowtot_item(const void *X, C *R, int64_t rows, int64_t L)
{
    LvItem w{};
    const int lpr = PM::row_lanes(L);
    w.kind = lpr <= 4 ? LV_RT_4 : lpr == 8 ? LV_RT_8 : lpr == 16 ? LV_RT_16 : LV_RT_32;
    w.src = X;
    w.r = R;
    w.O = rows;
    w.L = (int)L;
    const int64_t rpv = 4 * 4 * (32 / lpr);   // rows one sweep of a virtual block covers
    int64_t vg = std::min(cdiv64(rows, rpv), cdiv64(rows * L, 16384));
    w.vgrid = vg < 1 ? 1 : vg;
    w.vbase = 0;
    w.count = w.vgrid;
    return w;
}

struct Planned {
    std::vector<LvItem> items[NLV];
    size_t smem[NLV] = {};
    size_t bytes = 0;
};

// The window sums H1 along x1 (box k1 <= 32) of the lower problem's input
// (n1 planes of n2): a strided BDBS pass in the carry type, chunks sized as
// for the single-tensor pass.  Returns its level.
int h1_item(LvItem &w, const void *src, bool car, C *dst, int64_t n1, int64_t n2, int64_t k1, int sms)
{
    int Lc = 128;
    while (Lc > 2 * k1 && Lc > 16 && cdiv64(n1, Lc) * n2 < (int64_t)sms * 2048) Lc >>= 1;
    if (Lc > n1) Lc = (int)n1;
    w = LvItem{};
    w.kind = (car ? LV_H1C_K4 : LV_H1I_K4) + (k1 <= 4 ? 0 : k1 <= 8 ? 1 : k1 <= 16 ? 2 : 3);
    w.src = src;
    w.dst = dst;
    w.O = 1;
    w.n = (int)n1;
    w.I = n2;
    w.k = (int)k1;
    w.Lc = Lc;
    w.nchunks = (int)cdiv64(n1, Lc);
    w.vgrid = cdiv64((int64_t)w.nchunks * n2, 128);
    w.count = w.vgrid;
    return LV2H + lv_class(w.kind);
}

// Plans one tensor (accepted by level_accepts) into the level lists.
void plan_tensor(const exsum_desc &d, const LevelTune &tune, int sms, Carver &cv, Planned &pl)
{
    const int64_t *n = d.shape, *k = d.k;
    if (d.d == 2) {
        C *R2 = cv.take<C>(n[0]);
        C *H1 = k[0] > 1 ? cv.take<C>(n[0] * n[1]) : nullptr;
        LvItem p{};
        p.kind = LV_PT_IN;
        p.src = d.in;
        p.r = R2;
        p.n2 = (int)n[1];
        p.vgrid = n[0];
        p.count = n[0];
        pl.items[LV2].push_back(p);
        LvItem e{};
        e.kind = LV_E2_IN;
        e.src = d.in;
        if (H1) {
            // the window along x1 from a strided pass; the lower kernel reads one plane
            LvItem h;
            const int lv = h1_item(h, d.in, false, H1, n[0], n[1], k[0], sms);
            pl.items[lv].push_back(h);
            e.kind = LV_E2_CO;
            e.src = H1;
        }
        e.Lc = 1;   // planes combined per window by the lower kernel
        e.t = R2;
        e.dst = d.out;
        e.n = (int)n[0];
        e.n2 = (int)n[1];
        e.k = (int)k[0];
        e.k2 = (int)k[1];
        e.vgrid = cdiv64(n[0], 4);
        e.count = e.vgrid;
        pl.items[LV3].push_back(e);
        pl.smem[LV3] = std::max(pl.smem[LV3], 2 * 4 * (size_t)n[1] * sizeof(AccC));
        return;
    }
    const int64_t n0 = n[0], n1 = n[1], L = n[2], rows = n0 * n1, N = rows * L;
    // tall tiles: planned as if this tensor had the GPU to itself on one SM
    // (the tallest tile that fits), unless that loses the fused window
    auto rp = PM::row_plan(3, n, k, tune.tall ? 1 : sms);
    if (tune.tall) {
        const auto rs = PM::row_plan(3, n, k, sms);
        if (!rp.ok || rp.fuse != rs.fuse) rp = rs;
    }
    const bool s1 = k[0] > 1;
    const bool s2 = !rp.fuse && k[1] > 1;
    const int P = (int)s1 + (int)s2;
    Lt *B = P >= 1 ? cv.take<Lt>(N) : nullptr;
    Lt *B2 = P == 2 ? cv.take<Lt>(N) : nullptr;
    C *R = cv.take<C>(rows);
    C *T = cv.take<C>(rows);
    C *R2 = cv.take<C>(n0);
    C *H1 = k[0] > 1 ? cv.take<C>(rows) : nullptr;
    const void *X = d.in;

    // level 1: the strided pass along dimension 1 and the row totals
    if (s1) {
        Lt *dst = P == 1 ? B : B2;
        const int64_t I = n1 * L;
        const StridedPlan sp = strided_plan(X, dst, 1, n0, I, k[0], tune.lc, sms);
        if (tune.interleave) {
            // chunk c of the pass reads rows [c Lc, (c + 1) Lc) of dimension 1,
            // which hold the rows [c Lc n1, (c + 1) Lc n1) of R: their totals
            // go first (loads kept in L2), then the chunk's strided blocks
            for (int c = 0; c < sp.nchunks; ++c) {
                const int64_t r0 = (int64_t)c * sp.Lc * n1;
                const int64_t r1 = std::min(rows, (int64_t)(c + 1) * sp.Lc * n1);
                pl.items[LV1].push_back(rowtot_item(static_cast<const Lt *>(X) + r0 * L, R ? R + r0 : nullptr,
                                                    r1 - r0, L));
                const int64_t v0 = (int64_t)c * sp.per_chunk / 128;
                const int64_t v1 = c + 1 < sp.nchunks ? (int64_t)(c + 1) * sp.per_chunk / 128 : sp.vgrid;
                if (v1 > v0) pl.items[LV1 + lv_class(sp.kind)].push_back(strided_item(sp, X, dst, 1, n0, I, k[0], v0, v1));
            }
        } else {
            pl.items[LV1 + lv_class(sp.kind)].push_back(strided_item(sp, X, dst, 1, n0, I, k[0], 0, sp.vgrid));
            pl.items[LV1].push_back(rowtot_item(X, R, rows, L));
        }
    } else {
        pl.items[LV1].push_back(rowtot_item(X, R, rows, L));
    }
    // level 1b: the strided pass along dimension 2 when the final pass does not take it
    // (it reads the first pass's output, or X when there is no first pass)
    if (s2) {
        const void *src2 = s1 ? static_cast<const void *>(B2) : X;
        const StridedPlan sp = strided_plan(src2, B, n0, n1, L, k[1], tune.lc, sms);
        pl.items[(s1 ? LV1B : LV1) + lv_class(sp.kind)].push_back(strided_item(sp, src2, B, n0, n1, L, k[1], 0, sp.vgrid));
    }
    // levels 2 and 3: plane totals of R, then T = excluded(R)
    {
        LvItem p{};
        p.kind = LV_PT_CAR;
        p.src = R;
        p.r = R2;
        p.n2 = (int)n1;
        p.vgrid = n0;
        p.count = n0;
        pl.items[LV2].push_back(p);
        LvItem e{};
        e.kind = LV_E2_CAR;
        e.src = R;
        if (H1) {
            LvItem h;
            const int lv = h1_item(h, R, true, H1, n0, n1, k[0], sms);
            pl.items[lv].push_back(h);
            e.src = H1;
        }
        e.Lc = 1;
        e.t = R2;
        e.dst = T;
        e.n = (int)n0;
        e.n2 = (int)n1;
        e.k = (int)k[0];
        e.k2 = (int)k[1];
        e.vgrid = cdiv64(n0, 4);
        e.count = e.vgrid;
        pl.items[LV3].push_back(e);
        pl.smem[LV3] = std::max(pl.smem[LV3], 2 * 4 * (size_t)n1 * sizeof(AccC));
    }
    // level 4: the final pass
    const Lt *cur = P >= 1 ? B : static_cast<const Lt *>(X);
    const int kk = rp.fuse ? (int)k[1] : 1;
    const int k3 = (int)k[2];
    const bool bulk_ok = (!cv.base || al16(cur)) && al16(d.out) && L >= 128 && L <= 1024 &&
                         kk <= 32;
    if (bulk_ok) {
        const int kmax = kk <= 1 ? 1 : kk <= 8 ? 8 : 32;
        const auto bp = PM::bulk_plan(L, n1, n0, kk, kmax, sms, 2);
        if (bp.ok && bp.nbuf == 2 && bp.epl == 32 && bp.nt == 256 && bp.smem <= 113 * 1024) {
            LvItem w{};
            w.kind = kmax == 1 ? LV_BK_K1 : kmax == 8 ? LV_BK_K8 : LV_BK_K32;
            w.src = cur;
            w.t = T;
            w.dst = d.out;
            w.ntiles = bp.ntiles;
            w.ntile = bp.ntile;
            w.n2 = (int)n1;
            w.L = (int)L;
            w.k2 = kk;
            w.k3 = k3;
            w.TR = bp.TR;
            w.LSW = bp.LSW;
            w.lpr = bp.lpr;
            w.aligned = bp.aligned ? 1 : 0;
            const int tpv = tune.tiles_per_vb > 0 ? tune.tiles_per_vb : 2;
            w.vgrid = cdiv64(bp.ntiles, tpv);
            w.count = w.vgrid;
            const int lv4a = bp.odd ? LV4A_ODD : LV4A;
            pl.items[lv4a].push_back(w);
            pl.smem[lv4a] = std::max(pl.smem[lv4a], bp.smem);
            return;
        }
    }
    LvItem w{};
    const int base = kk <= 1 ? LV_RX_K1_E4 : kk <= 8 ? LV_RX_K8_E4 : LV_RX_K32_E4;
    w.kind = base + (rp.epl == 4 ? 0 : rp.epl == 8 ? 1 : rp.epl == 16 ? 2 : 3);
    w.src = cur;
    w.t = T;
    w.dst = d.out;
    w.O = n0;
    w.n2 = (int)n1;
    w.L = (int)L;
    w.k2 = kk;
    w.k3 = k3;
    w.TR = rp.TR;
    w.GO = rp.GO;
    w.ntile = rp.ntile;
    w.RS = rp.RS;
    w.RSA = rp.RSA;
    w.LS = rp.LS;
    w.lpr = rp.lpr;
    w.vgrid = cdiv64(n0, rp.GO) * rp.ntile;
    w.count = w.vgrid;
    const int lv4 = LV4B + lv_class(w.kind);
    pl.items[lv4].push_back(w);
    pl.smem[lv4] = std::max(pl.smem[lv4], rp.smem);
}

}  // namespace

namespace {

using KernFn = void (*)(LvList);

template <bool P>
KernFn level_kernel_t(int lv)
{
    switch (lv) {
    case LV1:
    case LV1B: return kl_stage1<M, 0, P>;
    case LV1_C1:
    case LV1B_C1: return kl_stage1<M, 1, P>;
    case LV2: return kl_plane<MC, P>;
    case LV2H: return kl_lower_h1<MC, 0, P>;
    case LV2H_C1: return kl_lower_h1<MC, 1, P>;
    case LV3: return kl_exc2d<MC, P>;
    case LV4A: return kl_final_bulk<M, P, false>;
    case LV4A_ODD: return kl_final_bulk<M, P, true>;
    case LV4B: return kl_final_rowx<M, 0, P>;
    case LV4B_C1: return kl_final_rowx<M, 1, P>;
    default: return kl_final_rowx<M, 2, P>;
    }
}

KernFn level_kernel(int lv, bool persist) { return persist ? level_kernel_t<true>(lv) : level_kernel_t<false>(lv); }

int64_t elems_of(const exsum_desc &d)
{
    int64_t n = 1;
    for (int i = 0; i < d.d; ++i) n *= d.shape[i];
    return n;
}

int cuda_fail(cudaError_t e)
{
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? EXSUM_ENOMEM : EXSUM_ECUDA;
}

}  // namespace

int level_create(const exsum_desc *descs, const int *idx, int n, const LevelTune &tune, LevelSet **out)
{
    *out = nullptr;
    if (n < 1) return EXSUM_EINVAL;
    const int sms = (int)device_sms();
    // largest tensor first: the small ones fill the tail of every launch
    std::vector<int> order(idx, idx + n);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return elems_of(descs[a]) > elems_of(descs[b]); });
    Carver sizing;
    {
        Planned dry;
        for (int t : order) plan_tensor(descs[t], tune, sms, sizing, dry);
    }
    LevelSet *ls = new LevelSet();
    ls->sms = sms;
    ls->persist = tune.persist != 0;
    ls->ws_bytes = sizing.off;
    auto fail = [&](int rc) {
        level_destroy(ls);
        return rc;
    };
    cudaError_t e = cudaSuccess;
    if (ls->ws_bytes) {
        e = cudaMalloc(&ls->ws, ls->ws_bytes);
        if (e != cudaSuccess) return fail(cuda_fail(e));
    }
    Carver cv;
    cv.base = static_cast<char *>(ls->ws);
    Planned pl;
    for (int t : order) plan_tensor(descs[t], tune, sms, cv, pl);
    // slot offsets and the slot -> item tables
    size_t total = 0, total_slots = 0;
    std::vector<int> slots;
    for (int lv = 0; lv < NLV; ++lv) {
        int64_t off = 0;
        int it = 0;
        for (LvItem &w : pl.items[lv]) {
            w.off = off;
            off += w.count;
            slots.insert(slots.end(), (size_t)w.count, it++);
        }
        if (off >= (1ll << 31)) return fail(EXSUM_EINVAL);
        ls->nslots[lv] = off;
        ls->item_base[lv] = total;
        ls->slot_base[lv] = total_slots;
        ls->smem[lv] = pl.smem[lv];
        total += pl.items[lv].size();
        total_slots += (size_t)off;
        ls->items[lv] = std::move(pl.items[lv]);
    }
    e = cudaMalloc(&ls->d_items, std::max<size_t>(total, 1) * sizeof(LvItem));
    if (e == cudaSuccess) e = cudaMalloc(&ls->d_slots, std::max<size_t>(total_slots, 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&ls->d_ctr, NLV * sizeof(unsigned long long));
    for (int lv = 0; lv < NLV && e == cudaSuccess; ++lv)
        if (!ls->items[lv].empty())
            e = cudaMemcpy(ls->d_items + ls->item_base[lv], ls->items[lv].data(),
                           ls->items[lv].size() * sizeof(LvItem), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && total_slots)
        e = cudaMemcpy(ls->d_slots, slots.data(), total_slots * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(cuda_fail(e));
    // grids: one block per slot, or (persistent) as many blocks as fit on
    // every SM at once
    for (int lv = 0; lv < NLV; ++lv) {
        if (!ls->nslots[lv]) continue;
        KernFn f = level_kernel(lv, ls->persist);
        if (ls->smem[lv] > 48 * 1024) {
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ls->smem[lv]);
            if (e != cudaSuccess) return fail(cuda_fail(e));
        }
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, kThreads[lv], ls->smem[lv]);
        if (e != cudaSuccess) return fail(cuda_fail(e));
        if (per_sm < 1) return fail(EXSUM_ENOMEM);
        const int64_t g = ls->persist ? (int64_t)sms * per_sm : ls->nslots[lv];
        ls->grid[lv] = (int)std::min<int64_t>(g, ls->nslots[lv]);
    }
    e = cudaStreamCreateWithFlags(&ls->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ls->side2, cudaStreamNonBlocking);
    for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ls->ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return fail(cuda_fail(e));
    *out = ls;
    return EXSUM_OK;
}

int level_enqueue(LevelSet *ls, cudaStream_t s)
{
    if (!ls) return EXSUM_EINVAL;
    cudaError_t e = cudaSuccess;
    if (ls->persist) {
        e = cudaMemsetAsync(ls->d_ctr, 0, NLV * sizeof(unsigned long long), s);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    auto has = [&](int lv) { return ls->nslots[lv] > 0; };
    auto launch = [&](int lv, cudaStream_t st) {
        if (!has(lv)) return;
        LvList l;
        l.items = ls->d_items + ls->item_base[lv];
        l.slot_item = ls->d_slots + ls->slot_base[lv];
        l.nslots = ls->nslots[lv];
        l.ctr = ls->persist ? ls->d_ctr + lv : nullptr;
        level_kernel(lv, ls->persist)<<<(unsigned)ls->grid[lv], (unsigned)kThreads[lv], ls->smem[lv], st>>>(l);
    };
    // runs a on s and b on the side stream, side by side (either may be empty)
    auto pair = [&](int a, int b) {
        if (has(a) && has(b)) {
            cudaEventRecord(ls->ev[0], s);
            cudaStreamWaitEvent(ls->side, ls->ev[0], 0);
            launch(b, ls->side);
            cudaEventRecord(ls->ev[1], ls->side);
            launch(a, s);
            cudaStreamWaitEvent(s, ls->ev[1], 0);
        } else {
            launch(a, s);
            launch(b, s);
        }
    };
    // level 1 (both register classes side by side)
    pair(LV1, LV1_C1);
    // level 1b (a second strided pass of some tensors) beside levels 2 and 3
    const bool b1 = has(LV1B) || has(LV1B_C1);
    if (b1) {
        cudaEventRecord(ls->ev[2], s);
        cudaStreamWaitEvent(ls->side, ls->ev[2], 0);
        launch(LV1B, ls->side);
        launch(LV1B_C1, ls->side);
        cudaEventRecord(ls->ev[3], ls->side);
    }
    // plane totals beside the window sums H1 (both read the lower input)
    const bool h1 = has(LV2H) || has(LV2H_C1);
    if (h1) {
        cudaEventRecord(ls->ev[4], s);
        cudaStreamWaitEvent(ls->side2, ls->ev[4], 0);
        launch(LV2H, ls->side2);
        launch(LV2H_C1, ls->side2);
        cudaEventRecord(ls->ev[5], ls->side2);
    }
    launch(LV2, s);
    if (h1) cudaStreamWaitEvent(s, ls->ev[5], 0);
    launch(LV3, s);
    if (b1) cudaStreamWaitEvent(s, ls->ev[3], 0);
    // the final-pass kernels side by side
    const int n4 = (int)has(LV4A) + (int)has(LV4A_ODD) + (int)has(LV4B) + (int)has(LV4B_C1) + (int)has(LV4B_C2);
    if (n4 > 1) {
        cudaEventRecord(ls->ev[4], s);
        cudaStreamWaitEvent(ls->side, ls->ev[4], 0);
        cudaStreamWaitEvent(ls->side2, ls->ev[4], 0);
        launch(LV4B, ls->side);
        launch(LV4B_C2, ls->side);
        launch(LV4B_C1, ls->side2);
        launch(LV4A, s);
        launch(LV4A_ODD, s);
        cudaEventRecord(ls->ev[5], ls->side);
        cudaStreamWaitEvent(s, ls->ev[5], 0);
        cudaEventRecord(ls->ev[1], ls->side2);
        cudaStreamWaitEvent(s, ls->ev[1], 0);
    } else {
        launch(LV4A, s);
        launch(LV4A_ODD, s);
        launch(LV4B, s);
        launch(LV4B_C1, s);
        launch(LV4B_C2, s);
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? EXSUM_OK : EXSUM_ECUDA;
}

size_t level_workspace_bytes(const LevelSet *ls) { return ls ? ls->ws_bytes : 0; }

int level_kernels(const LevelSet *ls)
{
    int c = 0;
    if (ls)
        for (int lv = 0; lv < NLV; ++lv) c += ls->nslots[lv] > 0;
    return c;
}

void level_destroy(LevelSet *ls)
{
    if (!ls) return;
    for (cudaEvent_t ev : ls->ev)
        if (ev) cudaEventDestroy(ev);
    if (ls->side) cudaStreamDestroy(ls->side);
    if (ls->side2) cudaStreamDestroy(ls->side2);
    if (ls->d_items) cudaFree(ls->d_items);
    if (ls->d_slots) cudaFree(ls->d_slots);
    if (ls->d_ctr) cudaFree(ls->d_ctr);
    if (ls->ws) cudaFree(ls->ws);
    delete ls;
}

}  // namespace exsum
