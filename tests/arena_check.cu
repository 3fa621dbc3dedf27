// arena_check.cu -- host-only check of the request server's device-memory
// arena (paper_2106_00124_gb300/csrc/exsum_server.cu): a first-fit allocator
// over one buffer, with free neighbours coalesced on release.  Random
// allocations and releases (a fixed-seed generator) run against a model
// that marks every 256-byte granule; after each step the check confirms
// that an allocation lies inside the arena on free granules, at the lowest
// offset of a free run that holds it (first fit), that an allocation fails
// only when no free run holds it (coalescing leaves no false shortage), and
// that releasing everything restores one block.  Prints "OK <steps>" or the
// first violations; test_arena.py runs it.  Nothing runs on a GPU: the
// library entry points the server calls are stubbed out below.
#include "../paper_2106_00124_gb300/csrc/exsum_server.cu"

#include <cstdio>
#include <vector>

// stand-ins for the library entry points the server file calls (never
// called here)
namespace exsum {
const void *aux_prepare(void *) { return nullptr; }
}
extern "C" {
size_t exsum_dtype_size(int) { return 0; }
int exsum_out_dtype(int) { return 0; }
size_t exsum_workspace_bytes(int, const int64_t *, const int64_t *, int, int, int, int *) { return 0; }
int exsum_excluded_ws(const void *, void *, int, const int64_t *, const int64_t *, int, int, void *, size_t, void *)
{
    return EXSUM_EINVAL;
}
}

namespace {

uint64_t g_state = 0x9e3779b97f4a7c15ull;
uint64_t next_u64()
{
    // splitmix64
    uint64_t z = (g_state += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

long g_bad = 0;
#define EXPECT(cond, ...)                   \
    do {                                    \
        if (!(cond)) {                      \
            if (g_bad < 20) {               \
                printf("V " __VA_ARGS__);   \
                printf(" [%s]\n", #cond);   \
            }                               \
            ++g_bad;                        \
        }                                   \
    } while (0)

constexpr size_t G = 256;

// first free run of the model holding n granules: its start, or -1
long first_fit(const std::vector<char> &used, size_t n)
{
    size_t run = 0;
    for (size_t i = 0; i < used.size(); ++i) {
        run = used[i] ? 0 : run + 1;
        if (run == n) return (long)(i + 1 - n);
    }
    return -1;
}

void run(size_t granules, int steps, int max_req)
{
    Arena a;
    a.reset(granules * G);
    std::vector<char> used(granules, 0);
    struct Live {
        size_t off, bytes;
    };
    std::vector<Live> live;
    for (int s = 0; s < steps; ++s) {
        const bool release = !live.empty() && (next_u64() % 100) < 45;
        if (release) {
            const size_t j = next_u64() % live.size();
            const Live l = live[j];
            live[j] = live.back();
            live.pop_back();
            a.release(l.off, l.bytes);
            const size_t n = l.bytes == 0 ? 1 : (l.bytes + G - 1) / G;
            for (size_t g = l.off / G; g < l.off / G + n; ++g) used[g] = 0;
            continue;
        }
        // sizes: zero, exact granules, ragged, and occasionally the whole arena
        size_t bytes;
        const uint64_t r = next_u64();
        if (r % 50 == 0)
            bytes = 0;
        else if (r % 97 == 1)
            bytes = granules * G;
        else if (r % 3 == 0)
            bytes = (1 + next_u64() % max_req) * G;
        else
            bytes = 1 + next_u64() % (max_req * G);
        const size_t n = bytes == 0 ? 1 : (bytes + G - 1) / G;
        const long want = first_fit(used, n);
        size_t off = 0;
        const bool ok = a.alloc(bytes, &off);
        EXPECT(ok == (want >= 0), "step %d: %zu bytes, allocated %d, a free run holds it %d", s, bytes, (int)ok,
               (int)(want >= 0));
        if (!ok) continue;
        EXPECT(off % G == 0 && off + n * G <= granules * G, "step %d: block [%zu, +%zu) outside the arena", s,
               off, n * G);
        EXPECT((long)(off / G) == want, "step %d: block at granule %zu, first fit at %ld", s, off / G, want);
        bool clash = false;
        for (size_t g = off / G; g < off / G + n && g < granules; ++g) {
            clash |= used[g] != 0;
            used[g] = 1;
        }
        EXPECT(!clash, "step %d: block [%zu, +%zu) overlaps a live block", s, off, n * G);
        live.push_back({off, bytes});
    }
    for (const Live &l : live) a.release(l.off, l.bytes);
    size_t off = 1;
    EXPECT(a.alloc(granules * G, &off) && off == 0, "all released: the arena is not one block again");
}

}  // namespace

int main()
{
    run(64, 20000, 8);        // small arena, frequent exhaustion
    run(4096, 20000, 300);    // larger blocks, fragmentation
    run(1, 2000, 1);          // one granule
    printf("%s %d\n", g_bad ? "BAD" : "OK", (int)g_bad);
    return g_bad ? 1 : 0;
}
