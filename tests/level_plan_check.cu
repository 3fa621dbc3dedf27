// level_plan_check.cu -- host-only check of the level planner
// (paper_2106_00124_gb300/csrc/exsum_level.cu): plans batches read from
// standard input with fake, well-separated device addresses and prints every
// work-list item with the fields the pass bodies index memory with.  The test
// (test_level_plan.py) checks that each item's reads and writes stay inside
// its tensor or the workspace.  Nothing runs on a GPU.
//
// Input: count, then per tensor "d n_1 .. n_d k_1 .. k_d"; environment LC,
// IL, TPV, TALL set the tuning, SKEW (bytes) moves every tensor off the
// 512-byte boundary its fake address otherwise starts on.
//
// Output lines: "S" element sizes, "K"/"L" the work-item kinds and levels by
// name, "T" one per tensor, "W" the workspace, "I" one per work item.
#include "../paper_2106_00124_gb300/csrc/exsum_level.cu"

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>

using namespace exsum;

// the pass kernels' wait-timeout counters register a reader with the C-ABI
// translation unit, which this program does not link
namespace exsum {
void register_timeout_reader(unsigned (*)()) {}
}

int main()
{
    int count = 0;
    if (scanf("%d", &count) != 1 || count < 1) return 1;
    const int skew = getenv("SKEW") ? atoi(getenv("SKEW")) : 0;
    printf("S %d %d\n", (int)sizeof(Lt), (int)sizeof(C));
#define NAME_KIND(x) printf("K %s %d\n", #x, (int)LV_##x)
    NAME_KIND(S4_K4); NAME_KIND(S4_K8); NAME_KIND(S1_K4); NAME_KIND(S1_K8); NAME_KIND(S1_K16);
    NAME_KIND(S1_K32); NAME_KIND(RT_4); NAME_KIND(RT_8); NAME_KIND(RT_16); NAME_KIND(RT_32);
    NAME_KIND(PT_IN); NAME_KIND(PT_CAR); NAME_KIND(E2_IN); NAME_KIND(E2_CAR); NAME_KIND(E2_CO);
    NAME_KIND(BK_K1); NAME_KIND(BK_K8); NAME_KIND(BK_K32);
    NAME_KIND(RX_K1_E4); NAME_KIND(RX_K1_E8); NAME_KIND(RX_K1_E16); NAME_KIND(RX_K1_E32);
    NAME_KIND(RX_K8_E4); NAME_KIND(RX_K8_E8); NAME_KIND(RX_K8_E16); NAME_KIND(RX_K8_E32);
    NAME_KIND(RX_K32_E4); NAME_KIND(RX_K32_E8); NAME_KIND(RX_K32_E16); NAME_KIND(RX_K32_E32);
    NAME_KIND(H1C_K4); NAME_KIND(H1C_K8); NAME_KIND(H1C_K16); NAME_KIND(H1C_K32);
    NAME_KIND(H1I_K4); NAME_KIND(H1I_K8); NAME_KIND(H1I_K16); NAME_KIND(H1I_K32);
#undef NAME_KIND
#define NAME_LEVEL(x) printf("L %s %d\n", #x, (int)x)
    NAME_LEVEL(LV1); NAME_LEVEL(LV1_C1); NAME_LEVEL(LV1B); NAME_LEVEL(LV1B_C1); NAME_LEVEL(LV2);
    NAME_LEVEL(LV2H); NAME_LEVEL(LV2H_C1); NAME_LEVEL(LV3); NAME_LEVEL(LV4A); NAME_LEVEL(LV4A_ODD);
    NAME_LEVEL(LV4B); NAME_LEVEL(LV4B_C1); NAME_LEVEL(LV4B_C2);
#undef NAME_LEVEL
    std::vector<exsum_desc> ds(count);
    std::vector<int> idx;
    uintptr_t next = 0x7f0000000000ull;
    for (int t = 0; t < count; ++t) {
        exsum_desc &d = ds[t];
        memset(&d, 0, sizeof(d));
        if (scanf("%d", &d.d) != 1) return 1;
        int64_t N = 1;
        for (int i = 0; i < d.d; ++i) {
            long long v;
            if (scanf("%lld", &v) != 1) return 1;
            d.shape[i] = v;
            N *= v;
        }
        for (int i = 0; i < d.d; ++i) {
            long long v;
            if (scanf("%lld", &v) != 1) return 1;
            d.k[i] = v;
        }
        d.op = EXSUM_OP_ADD;
        d.dtype = EXSUM_F32;
        d.in = (const void *)(next + skew);
        next += (N * 4 + skew + 511) / 512 * 512;
        d.out = (void *)(next + skew);
        next += (N * 4 + skew + 511) / 512 * 512;
        printf("T %d %llu %llu %lld %d\n", t, (unsigned long long)(uintptr_t)d.in,
               (unsigned long long)(uintptr_t)d.out, (long long)N, level_accepts(d, 152) ? 1 : 0);
        if (level_accepts(d, 152)) idx.push_back(t);
    }
    // largest tensor first, as the batch planner orders them
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
        int64_t na = 1, nb = 1;
        for (int i = 0; i < ds[a].d; ++i) na *= ds[a].shape[i];
        for (int i = 0; i < ds[b].d; ++i) nb *= ds[b].shape[i];
        return na > nb;
    });
    LevelTune tune;
    if (getenv("LC")) tune.lc = atoi(getenv("LC"));
    if (getenv("IL")) tune.interleave = atoi(getenv("IL"));
    if (getenv("TALL")) tune.tall = atoi(getenv("TALL"));
    if (getenv("TPV")) tune.tiles_per_vb = atoi(getenv("TPV"));
    Carver sizing;
    {
        Planned dry;
        for (int t : idx) plan_tensor(ds[t], tune, 152, sizing, dry);
    }
    const uintptr_t base = 0x100000000000ull;
    Carver cv;
    cv.base = (char *)base;
    Planned pl;
    for (int t : idx) plan_tensor(ds[t], tune, 152, cv, pl);
    printf("W %llu %llu %llu\n", (unsigned long long)base, (unsigned long long)sizing.off,
           (unsigned long long)cv.off);
    for (int lv = 0; lv < NLV; ++lv)
        for (const LvItem &w : pl.items[lv])
            printf("I %d %d %lld %lld %lld %llu %llu %llu %llu %lld %lld %d %d %d %d %d %d %d %d %d %d %d %d %d\n", lv,
                   w.kind, (long long)w.vbase, (long long)w.count, (long long)w.vgrid,
                   (unsigned long long)(uintptr_t)w.src, (unsigned long long)(uintptr_t)w.dst,
                   (unsigned long long)(uintptr_t)w.t, (unsigned long long)(uintptr_t)w.r, (long long)w.O,
                   (long long)w.I, w.n, w.k, w.Lc, w.nchunks, w.L, w.n2, w.k2, w.k3, w.TR, w.GO, w.ntile,
                   w.ntiles, w.lpr);
    return 0;
}
