// row_plan_check.cu -- host-only sweep of the final-pass planners of the row
// schedule (paper_2106_00124_gb300/csrc/pipeline.cuh): the tile plan of
// k_rowx (row_plan) and of the bulk-staged k_rowx_bulk (bulk_plan), for
// 4-byte (fp32 +) and 8-byte (int64 +) local types, over every row length
// the kernels take and a grid of slice heights, slice counts, windows and SM
// counts.  Each plan is checked against the conditions its kernel relies on:
// the shared memory it asks for fits a block and holds the tile, the tiles
// cover every row of a slice with none empty, the staged rows hold the
// window's halo, the strips of a row cover it, and the grid stays below
// 2^31 blocks.  Prints the counts and the first violations; the test
// (test_row_plan.py) asserts there are none.  Nothing runs on a GPU.
#include "../paper_2106_00124_gb300/csrc/pipeline.cuh"

#include <cstdio>

using namespace exsum;

namespace exsum {
void register_timeout_reader(unsigned (*)()) {}
}

namespace {

constexpr size_t kMaxSmem = 227 * 1024;   // dynamic shared memory a block may opt in to
long g_bad = 0;

#define EXPECT(cond, ...)                                      \
    do {                                                       \
        if (!(cond)) {                                         \
            if (g_bad < 20) {                                  \
                printf("V " __VA_ARGS__);                      \
                printf(" [%s]\n", #cond);                      \
            }                                                  \
            ++g_bad;                                           \
        }                                                      \
    } while (0)

int64_t cdivl(int64_t a, int64_t b) { return (a + b - 1) / b; }

template <class M>
void sweep_row_plan(const char *name, long &ok, long &refused)
{
    using PM = Pipe<M>;
    using L_ = typename PM::L_;
    using CAR = typename PM::CAR;
    const int64_t s = sizeof(L_);
    const int64_t lmax = s > 4 ? 512 : 1024;
    const int64_t n2s[] = {1, 2, 3, 7, 16, 33, 64, 76, 100, 256, 1000, 4096, 65536};
    const int64_t o2s[] = {1, 2, 5, 76, 1000, 65536, 1 << 22};
    const int64_t k2s[] = {1, 2, 4, 5, 8, 16, 31, 32, 33, 100};
    const int64_t smss[] = {152, 1};
    for (int64_t L = 16; L <= lmax; ++L)
        for (int64_t n2 : n2s)
            for (int64_t O2 : o2s)
                for (int64_t k2v : k2s)
                    for (int64_t sms : smss) {
                        const int64_t k2 = k2v < n2 ? k2v : n2;
                        const int64_t n[3] = {O2, n2, L};
                        const int64_t k[3] = {1, k2, 3};
                        const auto rp = PM::row_plan(3, n, k, sms);
                        if (!rp.ok) {
                            ++refused;
                            // every row length in range plans (the unfused tile
                            // of one row fits), unless the grid is too large
                            EXPECT(O2 * n2 >= (1ll << 31),
                                   "%s row_plan refused L=%lld n2=%lld O2=%lld k2=%lld sms=%lld", name,
                                   (long long)L, (long long)n2, (long long)O2, (long long)k2, (long long)sms);
                            continue;
                        }
                        ++ok;
                        const int64_t GO = rp.GO, TR = rp.TR, nt = rp.ntile;
                        const int64_t rpw = 32 / rp.lpr;
                        const int64_t L32 = cdivl(L, 32) * 32, LPs = L32 + 4 * (L32 / 32) + 4;
                        const int64_t tile = (GO * rp.RSA * rp.LS + (PM::ROWX_THREADS / 32) * rpw * LPs) * s;
#define ARGS name, (long long)L, (long long)n2, (long long)O2, (long long)k2, (long long)sms
                        EXPECT(rp.smem <= kMaxSmem, "%s smem L=%lld n2=%lld O2=%lld k2=%lld sms=%lld", ARGS);
                        EXPECT((int64_t)rp.smem >= tile + GO * TR * (int64_t)sizeof(CAR),
                               "%s smem below the tile L=%lld n2=%lld O2=%lld k2=%lld sms=%lld", ARGS);
                        EXPECT(GO >= 1 && GO <= O2 && (GO == 1 || GO * L <= PM::ROWX_THREADS),
                               "%s GO L=%lld n2=%lld O2=%lld k2=%lld sms=%lld", ARGS);
                        EXPECT(TR >= 1 && nt * TR >= n2 && (nt - 1) * TR < n2,
                               "%s tiles L=%lld n2=%lld O2=%lld k2=%lld sms=%lld", ARGS);
                        EXPECT(!rp.fuse || (k2 > 1 && k2 <= 32 && (nt == 1 || TR >= 2 * k2)),
                               "%s fused window L=%lld n2=%lld O2=%lld k2=%lld sms=%lld", ARGS);
                        EXPECT(rp.RS == (rp.fuse ? TR + k2 - 1 : TR) && rp.RSA >= rp.RS,
                               "%s staged rows L=%lld n2=%lld O2=%lld k2=%lld sms=%lld", ARGS);
                        EXPECT(rp.lpr >= 1 && rp.lpr <= 32 && (rp.lpr & (rp.lpr - 1)) == 0 &&
                                   (int64_t)rp.lpr * rp.epl >= L && (rp.epl == 4 || rp.epl == 8 || rp.epl == 16 ||
                                                                   (rp.epl == 32 && s == 4)),
                               "%s strips L=%lld n2=%lld O2=%lld k2=%lld sms=%lld", ARGS);
                        EXPECT(rp.LS >= cdivl(L, rp.epl) * rp.epl && (rp.LS * s) % 16 == 0,
                               "%s row stride L=%lld n2=%lld O2=%lld k2=%lld sms=%lld", ARGS);
                        EXPECT(cdivl(O2, GO) * nt < (1ll << 31), "%s grid L=%lld n2=%lld O2=%lld k2=%lld sms=%lld",
                               ARGS);
#undef ARGS
                    }
}

template <class M>
void sweep_bulk_plan(const char *name, long &ok, long &refused)
{
    using PM = Pipe<M>;
    const int64_t n2s[] = {1, 2, 3, 16, 33, 64, 100, 256, 1000, 65536};
    const int64_t o2s[] = {1, 3, 152, 4096, 1 << 20};
    const int kks[] = {1, 2, 3, 4, 5, 8, 9, 16, 17, 31, 32};
    for (int64_t L = 128; L <= 1024; ++L)
        for (int64_t n2 : n2s)
            for (int64_t O2 : o2s)
                for (int kk : kks) {
                    const int kmax = kk <= 1 ? 1 : kk <= 4 ? 4 : kk <= 8 ? 8 : kk <= 16 ? 16 : 32;
                    const auto bp = PM::bulk_plan(L, n2, O2, kk, kmax, 152);
                    if (!bp.ok) {
                        ++refused;
                        // without a window every row length plans, unless
                        // the tiles (at least 8 rows) would pass 2^31
                        EXPECT(kk > 1 || O2 * cdivl(n2, 8) >= (1ll << 31),
                               "%s bulk_plan refused L=%lld n2=%lld O2=%lld kk=%d", name, (long long)L,
                               (long long)n2, (long long)O2, kk);
                        continue;
                    }
                    ++ok;
#define ARGS name, (long long)L, (long long)n2, (long long)O2, kk
                    const int rows_pass = (bp.nt / 32) * (32 / bp.lpr);
                    const int G = rowbulk_segs((int)L, kmax, bp.nt, bp.odd);
                    EXPECT(bp.smem <= 226 * 1024, "%s bulk smem L=%lld n2=%lld O2=%lld kk=%d", ARGS);
                    EXPECT(bp.smem == rowbulk_smem(bp.TR, kk, bp.aligned, (int)L, bp.LSW, bp.nbuf, bp.odd),
                           "%s bulk smem formula L=%lld n2=%lld O2=%lld kk=%d", ARGS);
                    EXPECT(bp.TR >= rows_pass && bp.TR % rows_pass == 0,
                           "%s bulk tile height L=%lld n2=%lld O2=%lld kk=%d", ARGS);
                    EXPECT((int64_t)bp.lpr * bp.epl >= L && bp.LSW >= bp.lpr * bp.epl && bp.LSW % 32 == 0,
                           "%s bulk strips L=%lld n2=%lld O2=%lld kk=%d", ARGS);
                    EXPECT(bp.ntile == cdivl(n2, bp.TR) && (int64_t)bp.ntiles == O2 * bp.ntile,
                           "%s bulk tiles L=%lld n2=%lld O2=%lld kk=%d", ARGS);
                    EXPECT(bp.grid >= 1 && bp.grid <= bp.ntiles && bp.grid <= 2 * 152,
                           "%s bulk grid L=%lld n2=%lld O2=%lld kk=%d", ARGS);
                    EXPECT(!bp.aligned || (kk > 1 && bp.TR % G == 0 && (bp.TR / G) % kk == 0),
                           "%s bulk block-aligned walk L=%lld n2=%lld O2=%lld kk=%d", ARGS);
                    EXPECT(bp.odd == ((L & 3) != 0) && (!bp.odd || bp.nbuf == 2),
                           "%s bulk odd rows L=%lld n2=%lld O2=%lld kk=%d", ARGS);
#undef ARGS
                }
}

}  // namespace

int main()
{
    long ok = 0, refused = 0;
    sweep_row_plan<M_F32_ADD>("f32", ok, refused);
    printf("R f32 %ld %ld\n", ok, refused);
    ok = refused = 0;
    sweep_row_plan<M_I64_ADD>("i64", ok, refused);
    printf("R i64 %ld %ld\n", ok, refused);
    ok = refused = 0;
    sweep_bulk_plan<M_F32_ADD>("f32", ok, refused);
    printf("B f32 %ld %ld\n", ok, refused);
    printf("BAD %ld\n", g_bad);
    return 0;
}
