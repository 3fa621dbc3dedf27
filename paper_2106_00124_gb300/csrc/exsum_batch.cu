// exsum_batch.cu -- excluded sums of a batch of uneven tensors as one CUDA
// graph launch, with an autotuned schedule.
//
// A plan assigns the tensors of the batch to `lanes` concurrent streams
// (longest-processing-time first, or round-robin in size order), gives every
// lane one workspace sized for its largest tensor (a lane runs its tensors
// one after another, so they share it), and captures the whole batch --
// every pass of every tensor, with each tensor's own side-stream branches --
// into one CUDA graph that is launched with a single call.  The autotuner
// captures one graph per candidate schedule (lane counts 1..32, both
// orders), times a few replays of each and keeps the fastest; its choice is
// remembered per batch signature in memory and, when EXSUM_TUNE_CACHE names
// a file, across processes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/exsum.h"

namespace exsum {
const void *aux_prepare(void *stream);   // exsum_abi.cu: side streams of a caller stream
}

struct exsum_batch {
    int count = 0;
    int lanes = 0;
    int order = 0;                         // 0: LPT, 1: round-robin by size
    std::vector<exsum_desc> descs;
    std::vector<int> lane_of;              // tensor -> lane
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

std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tuned;   // signature -> (lanes, order)

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

void load_tune_file()
{
    static bool loaded = false;
    if (loaded) return;
    loaded = true;
    const char *path = getenv("EXSUM_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char key[64];
    int lanes, order;
    while (fscanf(f, "%63s %d %d", key, &lanes, &order) == 3) g_tuned[key] = {lanes, order};
    fclose(f);
}

void save_tune_entry(const std::string &key, int lanes, int order)
{
    const char *path = getenv("EXSUM_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d\n", key.c_str(), lanes, order);
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

// Assigns tensors to lanes and sizes the lane workspaces.
int schedule(exsum_batch *p, int lanes, int order)
{
    const int n = p->count;
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(),
                     [&](int a, int b) { return elems(p->descs[a]) > elems(p->descs[b]); });
    p->lanes = lanes;
    p->order = order;
    p->lane_items.assign(lanes, {});
    p->lane_of.assign(n, 0);
    std::vector<int64_t> load(lanes, 0);
    for (int j = 0; j < n; ++j) {
        const int t = idx[j];
        int lane;
        if (order == 0) {
            lane = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        } else {
            lane = j % lanes;
        }
        load[lane] += elems(p->descs[t]);
        p->lane_items[lane].push_back(t);
        p->lane_of[t] = lane;
    }
    p->lane_ws_bytes.assign(lanes, 0);
    for (int t = 0; t < n; ++t) {
        const exsum_desc &d = p->descs[t];
        int st = 0;
        const size_t b = exsum_workspace_bytes(d.d, d.shape, d.k, d.op, d.dtype, 1, &st);
        if (st) return st;
        size_t &m = p->lane_ws_bytes[p->lane_of[t]];
        m = std::max(m, b);
    }
    return EXSUM_OK;
}

// Allocates lane resources and captures the batch into a graph.
int build(exsum_batch *p)
{
    cudaError_t e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming);
    if (e != cudaSuccess) return EXSUM_ECUDA;
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
        cudaEventRecord(p->lane_join[l], p->lane_streams[l]);
        cudaStreamWaitEvent(p->cap, p->lane_join[l], 0);
    }
    e = cudaStreamEndCapture(p->cap, &p->graph);
    if (rc) return rc;
    if (e != cudaSuccess) return EXSUM_ECUDA;
    p->kernels = exsum_launch_count() - launches0;
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
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
}

}  // namespace

extern "C" {

int exsum_batch_create(const exsum_desc *descs, int count, int lanes, void *stream,
                       exsum_batch **plan)
{
    if (!plan || !descs || count < 1) return EXSUM_EINVAL;
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
    const std::string key = signature(descs, count);
    int order = 0;
    if (lanes <= 0) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        load_tune_file();
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            lanes = it->second.first;
            order = it->second.second;
        }
    }
    if (lanes <= 0) {
        // Autotune: capture each candidate schedule, time its replays, keep the best.
        float best = 3.4e38f;
        int best_lanes = 1, best_order = 0;
        const int cands[] = {1, 2, 4, 8, 16, 32};
        for (int c : cands) {
            if (c > count) break;
            for (int ord = 0; ord < 2; ++ord) {
                if (c == 1 && ord == 1) continue;
                exsum_batch trial;
                trial.count = count;
                trial.descs.assign(descs, descs + count);
                int rc = schedule(&trial, c, ord);
                if (!rc) rc = build(&trial);
                float ms = 3.4e38f;
                if (!rc) ms = time_replays(&trial, trial.cap, 3);
                release(&trial);
                if (rc == EXSUM_ENOMEM) continue;
                if (rc) return rc;
                if (ms < best) {
                    best = ms;
                    best_lanes = c;
                    best_order = ord;
                }
            }
        }
        lanes = best_lanes;
        order = best_order;
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tuned[key] = {lanes, order};
        save_tune_entry(key, lanes, order);
    }
    exsum_batch *p = new exsum_batch();
    p->count = count;
    p->descs.assign(descs, descs + count);
    int rc = schedule(p, std::min(lanes, count), order);
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
        size_t b = 0;
        for (size_t x : plan->lane_ws_bytes) b += x;
        *workspace_bytes = b;
    }
    if (kernels) *kernels = plan->kernels;
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
