// exsum_batch.cu -- excluded sums of a batch of uneven tensors as one CUDA
// graph launch, with an autotuned schedule.
//
// Two schedules.  Levels (exsum_level.cu): the tensors the level kernels
// take run as one launch per pass level (and register class), the rest on one lane
// beside it.  Lanes: the tensors are assigned to `lanes` concurrent streams
// (longest-processing-time first, or round-robin in size order), every lane
// gets one workspace sized for its largest tensor (a lane runs its tensors
// one after another, so they share it), and every pass of every tensor, with
// each tensor's own side-stream branches, is captured into the graph.  The
// autotuner captures one graph per candidate schedule, times a few replays
// of each and keeps the fastest; its choice is remembered per batch
// signature in memory and, when EXSUM_TUNE_CACHE names a file, across
// processes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/exsum.h"
#include "level.h"

namespace exsum {
const void *aux_prepare(void *stream);   // exsum_abi.cu: side streams of a caller stream
}

struct exsum_batch {
    int count = 0;
    int mode = 0;                          // 0: lanes, 1: levels
    int lanes = 0;
    int order = 0;                         // 0: LPT, 1: round-robin by size
    exsum::LevelTune tune;
    std::vector<exsum_desc> descs;
    std::vector<int> level_idx;            // tensors in the level set
    exsum::LevelSet *level = nullptr;
    std::vector<int> lane_of;              // tensor -> lane (-1: level set)
    std::vector<std::vector<int>> lane_items;
    std::vector<void *> lane_ws;
    std::vector<size_t> lane_ws_bytes;
    std::vector<cudaStream_t> lane_streams;
    std::vector<cudaEvent_t> lane_join;
    cudaEvent_t fork = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;
};

namespace {

// A schedule: mode, lanes/order (lanes mode, and the lane of the level
// mode's other tensors), level tuning.
struct Sched {
    int mode = 0, lanes = 1, order = 0;
    exsum::LevelTune tune;
};

std::mutex g_tune_mu;
std::map<std::string, Sched> g_tuned;   // signature -> schedule

std::string signature(const exsum_desc *descs, int count)
{
    // FNV-1a over the problem parameters (not the pointers)
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t v) {
        for (int i = 0; i < 8; ++i) {
            h ^= (v >> (8 * i)) & 0xff;
            h *= 1099511628211ull;
        }
    };
    mix((uint64_t)count);
    for (int t = 0; t < count; ++t) {
        mix((uint64_t)descs[t].d);
        mix((uint64_t)descs[t].op);
        mix((uint64_t)descs[t].dtype);
        for (int i = 0; i < descs[t].d; ++i) {
            mix((uint64_t)descs[t].shape[i]);
            mix((uint64_t)descs[t].k[i]);
        }
    }
    char buf[32];
    snprintf(buf, sizeof(buf), "%016llx", (unsigned long long)h);
    return buf;
}

// Cache file lines: "<signature> <mode> <lanes> <order> <lc> <interleave>
// <tiles_per_vb> <tall> <persist>"; lines of an older format (three fields:
// lanes schedules only) are read as lanes schedules.
void load_tune_file()
{
    static bool loaded = false;
    if (loaded) return;
    loaded = true;
    const char *path = getenv("EXSUM_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char line[256];
    while (fgets(line, sizeof(line), f)) {
        char key[64];
        Sched sc;
        int v[8];
        const int got = sscanf(line, "%63s %d %d %d %d %d %d %d %d", key, &v[0], &v[1], &v[2], &v[3], &v[4],
                               &v[5], &v[6], &v[7]);
        if (got == 9) {
            sc.mode = v[0];
            sc.lanes = v[1];
            sc.order = v[2];
            sc.tune.lc = v[3];
            sc.tune.interleave = v[4];
            sc.tune.tiles_per_vb = v[5];
            sc.tune.tall = v[6];
            sc.tune.persist = v[7];
        } else if (got == 3) {
            sc.mode = 0;
            sc.lanes = v[0];
            sc.order = v[1];
        } else {
            continue;
        }
        if (sc.lanes < 1) continue;
        g_tuned[key] = sc;
    }
    fclose(f);
}

void save_tune_entry(const std::string &key, const Sched &sc)
{
    const char *path = getenv("EXSUM_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d %d %d %d %d %d %d\n", key.c_str(), sc.mode, sc.lanes, sc.order, sc.tune.lc,
            sc.tune.interleave, sc.tune.tiles_per_vb, sc.tune.tall, sc.tune.persist);
    fclose(f);
}

int64_t elems(const exsum_desc &d)
{
    int64_t n = 1;
    for (int i = 0; i < d.d; ++i) n *= d.shape[i];
    return n;
}

void destroy_graph(exsum_batch *p)
{
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->exec = nullptr;
    p->graph = nullptr;
}

void release(exsum_batch *p)
{
    destroy_graph(p);
    exsum::level_destroy(p->level);
    p->level = nullptr;
    for (void *w : p->lane_ws)
        if (w) cudaFree(w);
    for (cudaEvent_t e : p->lane_join)
        if (e) cudaEventDestroy(e);
    for (cudaStream_t s : p->lane_streams)
        if (s) cudaStreamDestroy(s);
    if (p->fork) cudaEventDestroy(p->fork);
    if (p->cap) cudaStreamDestroy(p->cap);
    p->lane_ws.clear();
    p->lane_join.clear();
    p->lane_streams.clear();
    p->fork = nullptr;
    p->cap = nullptr;
}

// Splits the batch between the level set (level mode) and the lanes, assigns
// the lanes' tensors to lanes and sizes the lane workspaces.
int schedule(exsum_batch *p, const Sched &sc)
{
    const int n = p->count;
    p->mode = sc.mode;
    p->tune = sc.tune;
    p->order = sc.order;
    p->level_idx.clear();
    p->lane_of.assign(n, -1);
    std::vector<int> idx;
    for (int i = 0; i < n; ++i) {
        if (sc.mode == 1 && exsum::level_accepts(p->descs[i], exsum::level_sms()))
            p->level_idx.push_back(i);
        else
            idx.push_back(i);
    }
    const int lanes = std::max(1, std::min(sc.lanes, (int)idx.size()));
    std::stable_sort(idx.begin(), idx.end(),
                     [&](int a, int b) { return elems(p->descs[a]) > elems(p->descs[b]); });
    p->lanes = idx.empty() ? 0 : lanes;
    p->lane_items.assign(p->lanes, {});
    std::vector<int64_t> load(p->lanes, 0);
    for (size_t j = 0; j < idx.size(); ++j) {
        const int t = idx[j];
        int lane;
        if (sc.order == 0) {
            lane = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        } else {
            lane = (int)(j % p->lanes);
        }
        load[lane] += elems(p->descs[t]);
        p->lane_items[lane].push_back(t);
        p->lane_of[t] = lane;
    }
    p->lane_ws_bytes.assign(p->lanes, 0);
    for (int t : idx) {
        const exsum_desc &d = p->descs[t];
        int st = 0;
        const size_t b = exsum_workspace_bytes(d.d, d.shape, d.k, d.op, d.dtype, 1, &st);
        if (st) return st;
        size_t &m = p->lane_ws_bytes[p->lane_of[t]];
        m = std::max(m, b);
    }
    return EXSUM_OK;
}

// Allocates the plan's resources and captures the batch into a graph.
int build(exsum_batch *p)
{
    cudaError_t e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming);
    if (e != cudaSuccess) return EXSUM_ECUDA;
    if (!p->level_idx.empty()) {
        const int rc = exsum::level_create(p->descs.data(), p->level_idx.data(), (int)p->level_idx.size(), p->tune,
                                           &p->level);
        if (rc) return rc;
    }
    p->lane_streams.assign(p->lanes, nullptr);
    p->lane_join.assign(p->lanes, nullptr);
    p->lane_ws.assign(p->lanes, nullptr);
    for (int l = 0; l < p->lanes; ++l) {
        e = cudaStreamCreateWithFlags(&p->lane_streams[l], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->lane_join[l], cudaEventDisableTiming);
        if (e == cudaSuccess && p->lane_ws_bytes[l]) e = cudaMalloc(&p->lane_ws[l], p->lane_ws_bytes[l]);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? EXSUM_ENOMEM : EXSUM_ECUDA;
        }
        exsum::aux_prepare(p->lane_streams[l]);   // side streams, created outside capture
    }
    const int64_t launches0 = exsum_launch_count();
    e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return EXSUM_ECUDA;
    int rc = EXSUM_OK;
    cudaEventRecord(p->fork, p->cap);
    for (int l = 0; l < p->lanes && rc == EXSUM_OK; ++l) {
        cudaStreamWaitEvent(p->lane_streams[l], p->fork, 0);
        for (int t : p->lane_items[l]) {
            const exsum_desc &d = p->descs[t];
            rc = exsum_excluded_ws(d.in, d.out, d.d, d.shape, d.k, d.op, d.dtype, p->lane_ws[l],
                                   p->lane_ws_bytes[l], p->lane_streams[l]);
            if (rc) break;
        }
    }
    // the level set on the capture stream itself, beside the lanes
    if (rc == EXSUM_OK && p->level) rc = exsum::level_enqueue(p->level, p->cap);
    for (int l = 0; l < p->lanes; ++l) {
        cudaEventRecord(p->lane_join[l], p->lane_streams[l]);
        cudaStreamWaitEvent(p->cap, p->lane_join[l], 0);
    }
    e = cudaStreamEndCapture(p->cap, &p->graph);
    if (rc) return rc;
    if (e != cudaSuccess) return EXSUM_ECUDA;
    p->kernels = exsum_launch_count() - launches0 + exsum::level_kernels(p->level);
    // honour the per-node priorities of the side branches (see exsum_graph_instantiate)
    e = cudaGraphInstantiateWithFlags(&p->exec, p->graph, cudaGraphInstantiateFlagUseNodePriority);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return EXSUM_ECUDA;
    }
    return EXSUM_OK;
}

float time_replays(exsum_batch *p, cudaStream_t s, int reps)
{
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaGraphLaunch(p->exec, s);   // warm
    std::vector<float> t;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(a, s);
        cudaGraphLaunch(p->exec, s);
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        t.push_back(ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (cudaGetLastError() != cudaSuccess) return 3.4e38f;
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
}

// Builds and times one candidate; returns its median replay time in ms,
// or a huge value (rc set) if it could not be built.
float try_schedule(const exsum_desc *descs, int count, const Sched &sc, int *rc_out)
{
    exsum_batch trial;
    trial.count = count;
    trial.descs.assign(descs, descs + count);
    int rc = schedule(&trial, sc);
    if (!rc) rc = build(&trial);
    float ms = 3.4e38f;
    if (!rc) ms = time_replays(&trial, trial.cap, 3);
    release(&trial);
    *rc_out = rc;
    return ms;
}

// Autotuning: lanes schedules (1..32 lanes, both orders) and, when some
// tensors join a level set, level schedules by coordinate descent over the
// strided chunk length, the row-total placement, the bulk tiles per
// virtual block and the k_rowx tile height, from the defaults.
int autotune(const exsum_desc *descs, int count, Sched *best_out)
{
    float best = 3.4e38f;
    Sched best_sc;
    auto consider = [&](const Sched &sc) -> int {
        int rc = 0;
        const float ms = try_schedule(descs, count, sc, &rc);
        if (rc == EXSUM_ENOMEM) return EXSUM_OK;   // does not fit: skip
        if (rc) return rc;
        if (ms < best) {
            best = ms;
            best_sc = sc;
        }
        return EXSUM_OK;
    };
    const int cands[] = {1, 2, 4, 8, 16, 32};
    for (int c : cands) {
        if (c > count) break;
        for (int ord = 0; ord < 2; ++ord) {
            if (c == 1 && ord == 1) continue;
            Sched sc;
            sc.mode = 0;
            sc.lanes = c;
            sc.order = ord;
            const int rc = consider(sc);
            if (rc) return rc;
        }
    }
    int accepted = 0;
    for (int t = 0; t < count; ++t) accepted += exsum::level_accepts(descs[t], exsum::level_sms()) ? 1 : 0;
    if (accepted > 0) {
        Sched cur;
        cur.mode = 1;
        cur.lanes = std::min(4, std::max(1, count - accepted));
        float cur_ms = 3.4e38f;
        {
            const float b0 = best;
            const int rc = consider(cur);
            if (rc) return rc;
            if (best < b0) cur_ms = best;
        }
        // one field at a time, keeping each improvement
        auto step = [&](Sched s2) -> int {
            const float b0 = best;
            const int rc = consider(s2);
            if (rc) return rc;
            if (best < b0 && best < cur_ms) {
                cur = s2;
                cur_ms = best;
            }
            return EXSUM_OK;
        };
        const Sched base_lc = cur;
        for (int v : {32, 64, 128}) {
            Sched s2 = base_lc;
            s2.tune.lc = v;
            const int rc = step(s2);
            if (rc) return rc;
        }
        {
            Sched s2 = cur;
            s2.tune.interleave = 1 - cur.tune.interleave;
            const int rc = step(s2);
            if (rc) return rc;
        }
        const Sched base_tpv = cur;
        for (int v : {1, 4}) {
            Sched s2 = base_tpv;
            s2.tune.tiles_per_vb = v;
            const int rc = step(s2);
            if (rc) return rc;
        }
        {
            Sched s2 = cur;
            s2.tune.tall = 1 - cur.tune.tall;
            const int rc = step(s2);
            if (rc) return rc;
        }
        {
            Sched s2 = cur;
            s2.tune.persist = 1 - cur.tune.persist;
            const int rc = step(s2);
            if (rc) return rc;
        }
    }
    if (best >= 3.4e38f) return EXSUM_ENOMEM;
    *best_out = best_sc;
    return EXSUM_OK;
}

}  // namespace

extern "C" {

int exsum_batch_create(const exsum_desc *descs, int count, int lanes, void *stream,
                       exsum_batch **plan)
{
    if (!plan || !descs || count < 1 || lanes < EXSUM_BATCH_LEVELS) return EXSUM_EINVAL;
    *plan = nullptr;
    for (int t = 0; t < count; ++t) {
        const exsum_desc &d = descs[t];
        int st = 0;
        exsum_workspace_bytes(d.d, d.shape, d.k, d.op, d.dtype, 1, &st);
        if (st) return st;
        if (!d.in || !d.out) return EXSUM_EINVAL;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess ||
        cs != cudaStreamCaptureStatusNone)
        return EXSUM_EBUSY;
    Sched sc;
    if (lanes > 0) {
        sc.mode = 0;
        sc.lanes = lanes;
    } else if (lanes == EXSUM_BATCH_LEVELS) {
        sc.mode = 1;
        sc.lanes = 4;
        // EXSUM_LEVEL_TUNE="lc,interleave,tiles_per_vb,tall,persist" replaces the defaults
        if (const char *t = getenv("EXSUM_LEVEL_TUNE")) {
            int v[5];
            if (sscanf(t, "%d,%d,%d,%d,%d", &v[0], &v[1], &v[2], &v[3], &v[4]) == 5) {
                sc.tune.lc = v[0];
                sc.tune.interleave = v[1];
                sc.tune.tiles_per_vb = v[2];
                sc.tune.tall = v[3];
                sc.tune.persist = v[4];
            }
        }
    } else {
        const std::string key = signature(descs, count);
        bool found = false;
        {
            std::lock_guard<std::mutex> lock(g_tune_mu);
            load_tune_file();
            auto it = g_tuned.find(key);
            if (it != g_tuned.end()) {
                sc = it->second;
                found = true;
            }
        }
        if (!found) {
            const int rc = autotune(descs, count, &sc);
            if (rc) return rc;
            std::lock_guard<std::mutex> lock(g_tune_mu);
            g_tuned[key] = sc;
            save_tune_entry(key, sc);
        }
    }
    exsum_batch *p = new exsum_batch();
    p->count = count;
    p->descs.assign(descs, descs + count);
    int rc = schedule(p, sc);
    if (!rc) rc = build(p);
    if (rc) {
        release(p);
        delete p;
        return rc;
    }
    *plan = p;
    return EXSUM_OK;
}

int exsum_batch_launch(exsum_batch *plan, void *stream)
{
    if (!plan || !plan->exec) return EXSUM_EINVAL;
    cudaError_t e = cudaGraphLaunch(plan->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return EXSUM_ECUDA;
    }
    return EXSUM_OK;
}

int exsum_batch_info(const exsum_batch *plan, int *lanes, int *order, size_t *workspace_bytes,
                     int64_t *kernels)
{
    if (!plan) return EXSUM_EINVAL;
    if (lanes) *lanes = plan->lanes;
    if (order) *order = plan->order;
    if (workspace_bytes) {
        size_t b = exsum::level_workspace_bytes(plan->level);
        for (size_t x : plan->lane_ws_bytes) b += x;
        *workspace_bytes = b;
    }
    if (kernels) *kernels = plan->kernels;
    return EXSUM_OK;
}

int exsum_batch_schedule(const exsum_batch *plan, int *mode, int *level_tensors, int *lc, int *interleave,
                         int *tiles_per_vb, int *tall, int *persist)
{
    if (!plan) return EXSUM_EINVAL;
    if (mode) *mode = plan->mode;
    if (level_tensors) *level_tensors = (int)plan->level_idx.size();
    if (lc) *lc = plan->tune.lc;
    if (interleave) *interleave = plan->tune.interleave;
    if (tiles_per_vb) *tiles_per_vb = plan->tune.tiles_per_vb;
    if (tall) *tall = plan->tune.tall;
    if (persist) *persist = plan->tune.persist;
    return EXSUM_OK;
}

void exsum_batch_destroy(exsum_batch *plan)
{
    if (!plan) return;
    cudaDeviceSynchronize();
    release(plan);
    delete plan;
}

}  // extern "C"
