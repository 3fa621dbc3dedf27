// exsum_abi.cu -- the C ABI declared in include/exsum.h: argument checks,
// dtype/operator dispatch, and the per-(device, stream) workspace cache.
#include <cuda_runtime.h>

#include <atomic>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "../../include/exsum.h"
#include "pipeline.cuh"

namespace exsum {
int dispatch_i32(int, int, const void *, void *, int, const int64_t *, const int64_t *, void *,
                 size_t, cudaStream_t, size_t *, cudaError_t *, const Aux *);
int dispatch_i64(int, int, const void *, void *, int, const int64_t *, const int64_t *, void *,
                 size_t, cudaStream_t, size_t *, cudaError_t *, const Aux *);
int dispatch_f32(int, int, const void *, void *, int, const int64_t *, const int64_t *, void *,
                 size_t, cudaStream_t, size_t *, cudaError_t *, const Aux *);
int dispatch_bf16(int, int, const void *, void *, int, const int64_t *, const int64_t *, void *,
                  size_t, cudaStream_t, size_t *, cudaError_t *, const Aux *);
}  // namespace exsum

static thread_local int g_last_cuda_error = 0;

// ---- launch trace and launch counter --------------------------------------------------------
namespace {
struct TraceRec {
    int tag, level;
    int64_t elems;
    cudaEvent_t ev0, ev1;
};
std::atomic<int64_t> g_launches{0};
std::atomic<int64_t> g_side_streams{0};
std::atomic<int> g_trace_on{0};
std::mutex g_trace_mu;
std::vector<TraceRec> g_trace;
std::vector<cudaEvent_t> g_event_pool;
thread_local int g_pending = -1;

// Records ev on s; inside a stream capture the record becomes an event-record
// node of the graph (re-recorded on every replay).
void record_event(cudaEvent_t ev, cudaStream_t s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
    else
        cudaEventRecord(ev, s);
}

cudaEvent_t pool_event()
{
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}
}  // namespace

namespace exsum {
void trace_before(cudaStream_t s, int tag, int level, int64_t elems)
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    g_pending = -1;
    if (!g_trace_on.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lock(g_trace_mu);
    TraceRec r{tag, level, elems, pool_event(), pool_event()};
    if (!r.ev0 || !r.ev1) return;
    record_event(r.ev0, s);
    g_trace.push_back(r);
    g_pending = (int)g_trace.size() - 1;
}

void trace_after(cudaStream_t s)
{
    if (g_pending < 0) return;
    std::lock_guard<std::mutex> lock(g_trace_mu);
    if (g_pending < (int)g_trace.size()) record_event(g_trace[g_pending].ev1, s);
    g_pending = -1;
}
}  // namespace exsum

static int validate(int d, const int64_t *shape, const int64_t *k, int op, int dtype)
{
    if (d < 1 || d > EXSUM_MAX_DIMS || !shape || !k) return EXSUM_EINVAL;
    if (op != EXSUM_OP_ADD && op != EXSUM_OP_MAX) return EXSUM_EINVAL;
    if (dtype < EXSUM_I32 || dtype > EXSUM_BF16) return EXSUM_EINVAL;
    int64_t N = 1;
    for (int i = 0; i < d; ++i) {
        if (shape[i] < 1 || k[i] < 1 || k[i] > shape[i]) return EXSUM_EINVAL;
        if (N > ((int64_t)1 << 62) / shape[i]) return EXSUM_EINVAL;  // element count overflow
        N *= shape[i];
    }
    return EXSUM_OK;
}

// ---- side streams: one (stream, fork event, join event) per (device, caller stream) -------------
namespace {
std::mutex g_aux_mu;
std::map<std::pair<int, void *>, exsum::Aux> g_aux;
}  // namespace

// The side stream of the caller's stream, created on first use outside any
// stream capture; nullptr (run everything on the caller's stream) otherwise.
static const exsum::Aux *aux_for(void *stream)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_aux_mu);
    auto key = std::make_pair(dev, stream);
    auto it = g_aux.find(key);
    if (it != g_aux.end()) return it->second.side ? &it->second : nullptr;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess ||
        cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return nullptr;
    }
    // The side branches are chains of short kernels on the critical path,
    // launched while the caller's stream runs a full-tensor pass: the highest
    // stream priority lets their blocks take SM slots as the pass's blocks
    // retire.  (Graphs keep it per node; cudaGraphInstantiateFlagUseNodePriority
    // honours it, see exsum_graph_instantiate.)
    exsum::Aux a;
    int lo = 0, hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) {
        cudaGetLastError();
        hi = 0;
    }
    if (cudaStreamCreateWithPriority(&a.side, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&a.side2, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&a.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&a.join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&a.fork2, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&a.join2, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        a = exsum::Aux();
    }
    if (a.side) g_side_streams.fetch_add(2);
    g_aux[key] = a;
    return a.side ? &g_aux[key] : nullptr;
}

namespace exsum {
// Creates (outside any capture) the side streams of a caller stream, so that
// later calls on that stream fork even while it is being captured.
const void *aux_prepare(void *stream) { return aux_for(stream); }
}  // namespace exsum

static int run(int excluded, const void *in, void *out, int d, const int64_t *shape,
               const int64_t *k, int op, int dtype, void *ws, size_t ws_bytes, void *stream,
               size_t *need, bool allow_fork = true)
{
    cudaError_t ce = cudaSuccess;
    int rc;
    cudaStream_t st = (cudaStream_t)stream;
    const exsum::Aux *aux = (in && excluded && allow_fork) ? aux_for(stream) : nullptr;
    switch (dtype) {
    case EXSUM_I32: rc = exsum::dispatch_i32(op, excluded, in, out, d, shape, k, ws, ws_bytes, st, need, &ce, aux); break;
    case EXSUM_I64: rc = exsum::dispatch_i64(op, excluded, in, out, d, shape, k, ws, ws_bytes, st, need, &ce, aux); break;
    case EXSUM_F32: rc = exsum::dispatch_f32(op, excluded, in, out, d, shape, k, ws, ws_bytes, st, need, &ce, aux); break;
    default: rc = exsum::dispatch_bf16(op, excluded, in, out, d, shape, k, ws, ws_bytes, st, need, &ce, aux); break;
    }
    if (rc == EXSUM_ECUDA) g_last_cuda_error = (int)ce;
    return rc;
}

// ---- workspace cache: one growing buffer per (device, stream) --------------------------------
namespace {
struct CacheEntry {
    void *ptr = nullptr;
    size_t bytes = 0;
};
std::mutex g_cache_mu;
std::map<std::pair<int, void *>, CacheEntry> g_cache;
}  // namespace

static int cached_workspace(void *stream, size_t need, void **ws, size_t *ws_bytes)
{
    *ws = nullptr;
    *ws_bytes = 0;
    if (need == 0) return EXSUM_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        g_last_cuda_error = (int)e;
        return EXSUM_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_cache_mu);
    CacheEntry &ent = g_cache[std::make_pair(dev, stream)];
    if (ent.bytes < need) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        e = cudaStreamIsCapturing((cudaStream_t)stream, &cs);
        if (e != cudaSuccess) {
            g_last_cuda_error = (int)e;
            return EXSUM_ECUDA;
        }
        if (cs != cudaStreamCaptureStatusNone) return EXSUM_EBUSY;
        if (ent.ptr) {
            // Earlier work on this stream may still use the old buffer.
            e = cudaStreamSynchronize((cudaStream_t)stream);
            if (e == cudaSuccess) e = cudaFree(ent.ptr);
            ent.ptr = nullptr;
            ent.bytes = 0;
            if (e != cudaSuccess) {
                g_last_cuda_error = (int)e;
                return EXSUM_ECUDA;
            }
        }
        const size_t grow = need + need / 4;
        e = cudaMalloc(&ent.ptr, grow);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ent.ptr = nullptr;
            g_last_cuda_error = (int)e;
            return EXSUM_ENOMEM;
        }
        ent.bytes = grow;
    }
    *ws = ent.ptr;
    *ws_bytes = ent.bytes;
    return EXSUM_OK;
}

static int call_cached(int excluded, const void *in, void *out, int d, const int64_t *shape,
                       const int64_t *k, int op, int dtype, void *stream)
{
    int rc = validate(d, shape, k, op, dtype);
    if (rc) return rc;
    if (!in || !out) return EXSUM_EINVAL;
    size_t need = 0;
    rc = run(excluded, nullptr, nullptr, d, shape, k, op, dtype, nullptr, 0, nullptr, &need);
    if (rc) return rc;
    void *ws = nullptr;
    size_t wsb = 0;
    rc = cached_workspace(stream, need, &ws, &wsb);
    if (rc) return rc;
    return run(excluded, in, out, d, shape, k, op, dtype, ws, wsb, stream, nullptr);
}

// ---- weak excluded sums (total minus included; integer + only) ------------------------------
namespace {
// Total of the tensor modulo 2^64 (the low 32 bits are the int32 total
// modulo 2^32): warp sums of a grid-stride walk, added atomically.
template <class T>
__global__ void __launch_bounds__(256) k_weak_total(const T *__restrict__ x, int64_t n,
                                                     unsigned long long *__restrict__ acc)
{
    unsigned long long s = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        s += (unsigned long long)(long long)x[i];
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
    if ((threadIdx.x & 31) == 0) atomicAdd(acc, s);
}

// out[i] = total - out[i], wrapping.
template <class T, class U>
__global__ void __launch_bounds__(256) k_weak_finish(T *__restrict__ out, int64_t n,
                                                      const unsigned long long *__restrict__ acc)
{
    const U tot = (U)*acc;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = (T)(tot - (U)out[i]);
}

template <class T, class U>
int weak_launch(const void *in, void *out, int64_t N, unsigned long long *acc, cudaStream_t st)
{
    int sms = 152, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (N + 255) / 256;
    if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
    if (blocks < 1) blocks = 1;
    exsum::trace_before(st, exsum::TAG_WEAK, 0, N);
    k_weak_finish<T, U><<<(unsigned)blocks, 256, 0, st>>>((T *)out, N, acc);
    exsum::trace_after(st);
    (void)in;
    return EXSUM_OK;
}
}  // namespace

extern "C" {

int exsum_version(void) { return 10000; }

const char *exsum_strerror(int status)
{
    switch (status) {
    case EXSUM_OK: return "success";
    case EXSUM_EINVAL: return "invalid argument";
    case EXSUM_ENOMEM: return "workspace too small or allocation failed";
    case EXSUM_EUNSUPPORTED: return "unsupported request";
    case EXSUM_ECUDA: return "CUDA runtime error";
    case EXSUM_ETIMEDOUT: return "timed out";
    case EXSUM_EBUSY: return "busy";
    default: return "unknown status";
    }
}

int exsum_last_cuda_error(void) { return g_last_cuda_error; }

int exsum_out_dtype(int dtype)
{
    if (dtype < EXSUM_I32 || dtype > EXSUM_BF16) return -1;
    return dtype == EXSUM_BF16 ? EXSUM_F32 : dtype;
}

size_t exsum_dtype_size(int dtype)
{
    switch (dtype) {
    case EXSUM_I32: return 4;
    case EXSUM_I64: return 8;
    case EXSUM_F32: return 4;
    case EXSUM_BF16: return 2;
    default: return 0;
    }
}

size_t exsum_workspace_bytes(int d, const int64_t *shape, const int64_t *k, int op, int dtype,
                             int excluded, int *status)
{
    int rc = validate(d, shape, k, op, dtype);
    size_t need = 0;
    if (!rc) rc = run(excluded ? 1 : 0, nullptr, nullptr, d, shape, k, op, dtype, nullptr, 0, nullptr, &need);
    if (status) *status = rc;
    return rc ? 0 : need;
}

int exsum_excluded_weak(const void *in, void *out, int d, const int64_t *shape, const int64_t *k,
                        int dtype, void *stream)
{
    int rc = validate(d, shape, k, EXSUM_OP_ADD, dtype);
    if (rc) return rc;
    if (dtype != EXSUM_I32 && dtype != EXSUM_I64) return EXSUM_EUNSUPPORTED;
    if (!in || !out) return EXSUM_EINVAL;
    int64_t N = 1;
    for (int i = 0; i < d; ++i) N *= shape[i];
    size_t need = 0;
    rc = run(0, nullptr, nullptr, d, shape, k, EXSUM_OP_ADD, dtype, nullptr, 0, nullptr, &need);
    if (rc) return rc;
    const size_t inc_bytes = (need + 255) & ~(size_t)255;
    void *ws = nullptr;
    size_t wsb = 0;
    rc = cached_workspace(stream, inc_bytes + 256, &ws, &wsb);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long *acc = (unsigned long long *)((char *)ws + inc_bytes);
    cudaError_t ce = cudaMemsetAsync(acc, 0, sizeof(*acc), st);
    if (ce == cudaSuccess) {
        int sms = 152, dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess)
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        int64_t blocks = (N + 255) / 256;
        if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
        exsum::trace_before(st, exsum::TAG_REDUCE, 0, N);
        if (dtype == EXSUM_I32)
            k_weak_total<int32_t><<<(unsigned)blocks, 256, 0, st>>>((const int32_t *)in, N, acc);
        else
            k_weak_total<int64_t><<<(unsigned)blocks, 256, 0, st>>>((const int64_t *)in, N, acc);
        exsum::trace_after(st);
        ce = cudaGetLastError();
    }
    if (ce != cudaSuccess) {
        g_last_cuda_error = (int)ce;
        return EXSUM_ECUDA;
    }
    rc = run(0, in, out, d, shape, k, EXSUM_OP_ADD, dtype, ws, inc_bytes, stream, nullptr);
    if (rc) return rc;
    if (dtype == EXSUM_I32)
        weak_launch<int32_t, uint32_t>(in, out, N, acc, st);
    else
        weak_launch<int64_t, uint64_t>(in, out, N, acc, st);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        g_last_cuda_error = (int)ce;
        return EXSUM_ECUDA;
    }
    return EXSUM_OK;
}

int exsum_included(const void *in, void *out, int d, const int64_t *shape, const int64_t *k, int op,
                   int dtype, void *stream)
{
    return call_cached(0, in, out, d, shape, k, op, dtype, stream);
}

int exsum_excluded(const void *in, void *out, int d, const int64_t *shape, const int64_t *k, int op,
                   int dtype, void *stream)
{
    return call_cached(1, in, out, d, shape, k, op, dtype, stream);
}

int exsum_included_ws(const void *in, void *out, int d, const int64_t *shape, const int64_t *k,
                      int op, int dtype, void *workspace, size_t workspace_bytes, void *stream)
{
    int rc = validate(d, shape, k, op, dtype);
    if (rc) return rc;
    if (!in || !out) return EXSUM_EINVAL;
    return run(0, in, out, d, shape, k, op, dtype, workspace, workspace_bytes, stream, nullptr);
}

int exsum_excluded_ws(const void *in, void *out, int d, const int64_t *shape, const int64_t *k,
                      int op, int dtype, void *workspace, size_t workspace_bytes, void *stream)
{
    int rc = validate(d, shape, k, op, dtype);
    if (rc) return rc;
    if (!in || !out) return EXSUM_EINVAL;
    return run(1, in, out, d, shape, k, op, dtype, workspace, workspace_bytes, stream, nullptr);
}

void exsum_trace_enable(int on) { g_trace_on.store(on ? 1 : 0); }

int exsum_trace_collect(int *tags, int *levels, int64_t *elems, float *ms, int cap, int clear)
{
    std::lock_guard<std::mutex> lock(g_trace_mu);
    int n = 0;
    int rc = 0;
    for (auto &r : g_trace) {
        float t = -1.f;
        cudaError_t e = cudaEventSynchronize(r.ev1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.ev0, r.ev1);
        if (e != cudaSuccess) {
            g_last_cuda_error = (int)e;
            cudaGetLastError();
            rc = EXSUM_ECUDA;
        }
        if (n < cap) {
            if (tags) tags[n] = r.tag;
            if (levels) levels[n] = r.level;
            if (elems) elems[n] = r.elems;
            if (ms) ms[n] = t;
        }
        ++n;
        if (clear) {
            g_event_pool.push_back(r.ev0);
            g_event_pool.push_back(r.ev1);
        }
    }
    if (clear) g_trace.clear();
    return rc ? rc : n;
}

const char *exsum_kernel_name(int tag)
{
    switch (tag) {
    case exsum::TAG_INC: return "bdbs_along_dim_lines";
    case exsum::TAG_INC_CONTIG: return "bdbs_along_dim_contiguous";
    case exsum::TAG_INC_STRIDED: return "bdbs_along_dim_strided";
    case exsum::TAG_REDUCE: return "segment_reduce";
    case exsum::TAG_SUMSEG: return "segment_totals";
    case exsum::TAG_CARRY: return "dim1_carries";
    case exsum::TAG_EXLINE: return "dim1_prefix_suffix_contrib";
    case exsum::TAG_ROWSUM: return "row_totals";
    case exsum::TAG_ROWX: return "row_prefix_suffix_contrib";
    case exsum::TAG_WEAK: return "weak_total_minus_included";
    case exsum::TAG_INC_FOLD: return "bdbs_along_dim_strided_row_totals";
    case exsum::TAG_PLANE: return "plane_totals";
    case exsum::TAG_EXC2D: return "excluded_2d_lower";
    default: return "unknown";
    }
}

int64_t exsum_launch_count(void) { return g_launches.load(); }

int64_t exsum_side_streams_created(void) { return g_side_streams.load(); }

int exsum_graph_instantiate(void *graph, void **exec)
{
    if (!graph || !exec) return EXSUM_EINVAL;
    cudaGraphExec_t e = nullptr;
    const cudaError_t ce = cudaGraphInstantiateWithFlags(&e, (cudaGraph_t)graph,
                                                         cudaGraphInstantiateFlagUseNodePriority);
    if (ce != cudaSuccess) {
        g_last_cuda_error = (int)ce;
        cudaGetLastError();
        *exec = nullptr;
        return EXSUM_ECUDA;
    }
    *exec = (void *)e;
    return EXSUM_OK;
}

int exsum_graph_launch(void *exec, void *stream)
{
    if (!exec) return EXSUM_EINVAL;
    const cudaError_t ce = cudaGraphLaunch((cudaGraphExec_t)exec, (cudaStream_t)stream);
    if (ce != cudaSuccess) {
        g_last_cuda_error = (int)ce;
        cudaGetLastError();
        return EXSUM_ECUDA;
    }
    return EXSUM_OK;
}

int exsum_graph_exec_destroy(void *exec)
{
    if (!exec) return EXSUM_EINVAL;
    const cudaError_t ce = cudaGraphExecDestroy((cudaGraphExec_t)exec);
    if (ce != cudaSuccess) {
        g_last_cuda_error = (int)ce;
        cudaGetLastError();
        return EXSUM_ECUDA;
    }
    return EXSUM_OK;
}

}  // extern "C"

namespace exsum {
// Readers of the per-translation-unit counters of bulk-copy waits that gave
// up (kernels_rowbulk.cuh), registered at load time.
static std::vector<unsigned (*)()> &timeout_readers()
{
    static std::vector<unsigned (*)()> v;
    return v;
}
void register_timeout_reader(unsigned (*reader)()) { timeout_readers().push_back(reader); }

// For the other translation units (exsum_cmp.cu): argument checks and the
// cached per-stream workspace.
int validate_args(int d, const int64_t *shape, const int64_t *k, int op, int dtype)
{
    return validate(d, shape, k, op, dtype);
}
int cached_ws(void *stream, size_t need, void **ws, size_t *bytes) { return cached_workspace(stream, need, ws, bytes); }

// exsum_excluded_ws without the side stream: everything on `stream`, no
// stream or event is ever created (used by the allocation-free entry point).
int excluded_ws_serial(const void *in, void *out, int d, const int64_t *shape, const int64_t *k,
                       int op, int dtype, void *workspace, size_t workspace_bytes, void *stream)
{
    int rc = validate(d, shape, k, op, dtype);
    if (rc) return rc;
    if (!in || !out) return EXSUM_EINVAL;
    return run(1, in, out, d, shape, k, op, dtype, workspace, workspace_bytes, stream, nullptr,
               false);
}
}  // namespace exsum

extern "C" {

unsigned exsum_device_timeouts(void)
{
    unsigned total = 0;
    for (auto f : exsum::timeout_readers()) total += f();
    return total;
}

int exsum_release_cached_workspace(void)
{
    std::lock_guard<std::mutex> lock(g_cache_mu);
    cudaError_t e = cudaDeviceSynchronize();
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &kv : g_cache) {
        if (kv.second.ptr) {
            cudaSetDevice(kv.first.first);
            cudaError_t f = cudaFree(kv.second.ptr);
            if (e == cudaSuccess) e = f;
        }
    }
    cudaSetDevice(cur);
    g_cache.clear();
    if (e != cudaSuccess) {
        g_last_cuda_error = (int)e;
        return EXSUM_ECUDA;
    }
    return EXSUM_OK;
}

}  // extern "C"
