// exsum_server.cu -- a continuous-batching request server for excluded sums.
//
// Requests (one excluded sum each, any shape / box / operator / dtype) are
// queued by exsum_server_submit and admitted in arrival order by a host
// worker thread as soon as (a) a slot -- one CUDA stream -- is free and (b)
// the request's device memory fits in the server's budget.  Admitted
// requests run concurrently on their slots while later ones keep arriving;
// their state (workspace and, for host-pointer requests, staged input and
// output) lives in one device arena allocated once at creation, so serving
// allocates nothing.  Completion is signalled from the stream itself (a host
// function enqueued after the request's work), which frees the request's
// arena blocks and wakes the worker and any waiter.  Waits take a timeout and
// return EXSUM_ETIMEDOUT instead of blocking forever.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/exsum.h"

namespace exsum {
const void *aux_prepare(void *stream);
}

namespace {

int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// First-fit allocator over [0, size) with coalescing of free neighbours.
class Arena {
public:
    void reset(size_t size)
    {
        free_.clear();
        if (size) free_[0] = size;
    }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = (bytes + 255) & ~(size_t)255;
        if (bytes == 0) bytes = 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = (bytes + 255) & ~(size_t)255;
        if (bytes == 0) bytes = 256;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }

private:
    std::map<size_t, size_t> free_;
};

struct Request {
    uint64_t ticket = 0;
    exsum_desc desc{};
    int flags = 0;
    size_t ws_bytes = 0, in_bytes = 0, out_bytes = 0;
    size_t need = 0;                 // arena bytes
    size_t off = 0;                  // arena offset
    int slot = -1;
    int status = EXSUM_OK;
    bool done = false;
    int64_t t_submit = 0, t_start = 0, t_done = 0;
    int64_t not_before = 0;          // arrival time: not admitted earlier
};

}  // namespace

struct exsum_server {
    int device = 0;
    size_t budget = 0;
    char *arena_base = nullptr;
    Arena arena;
    std::vector<cudaStream_t> slots;
    std::vector<int> slot_busy;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Request> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    int64_t completed = 0;
    int fail_next = 0;               // host-side fault injection (exsum_server_fail_next)
    int fail_status = EXSUM_OK;
};

namespace {

// What the stream-ordered callback needs: the request, and the status it
// ends with (a failed launch passes its error here, so that `done` and
// `status` change together under the lock).
struct Completion {
    exsum_server *srv;
    uint64_t ticket;
    int status;
};

void CUDART_CB on_complete(void *data)
{
    Completion *c = static_cast<Completion *>(data);
    exsum_server *srv = c->srv;
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        auto it = srv->reqs.find(c->ticket);
        if (it != srv->reqs.end()) {
            Request &r = it->second;
            srv->arena.release(r.off, r.need);
            srv->slot_busy[r.slot] = 0;
            if (c->status != EXSUM_OK) r.status = c->status;
            r.done = true;
            r.t_done = now_ns();
            srv->completed++;
        }
    }
    srv->cv_work.notify_one();
    srv->cv_done.notify_all();
    delete c;
}

// Enqueues an admitted request on its slot (called without the lock).
int launch(exsum_server *srv, Request &r)
{
    cudaStream_t s = srv->slots[r.slot];
    char *base = srv->arena_base + r.off;
    char *ws = base;
    const void *in = r.desc.in;
    void *out = r.desc.out;
    if (r.flags & EXSUM_SERVE_HOST) {
        char *din = base + ((r.ws_bytes + 255) & ~(size_t)255);
        char *dout = din + ((r.in_bytes + 255) & ~(size_t)255);
        if (cudaMemcpyAsync(din, r.desc.in, r.in_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return EXSUM_ECUDA;
        in = din;
        out = dout;
    }
    int rc = exsum_excluded_ws(in, out, r.desc.d, r.desc.shape, r.desc.k, r.desc.op, r.desc.dtype,
                               ws, r.ws_bytes, s);
    if (rc) return rc;
    if (r.flags & EXSUM_SERVE_HOST) {
        if (cudaMemcpyAsync(r.desc.out, out, r.out_bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return EXSUM_ECUDA;
    }
    Completion *c = new Completion{srv, r.ticket, EXSUM_OK};
    if (cudaLaunchHostFunc(s, on_complete, c) != cudaSuccess) {
        delete c;
        return EXSUM_ECUDA;
    }
    return EXSUM_OK;
}

void worker_main(exsum_server *srv)
{
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lock(srv->mu);
    while (true) {
        // Admit in arrival order while a slot is free and the head fits.  The
        // lock is held only for the bookkeeping: CUDA calls are made without
        // it, because the completion callback running on CUDA's own thread
        // takes it.
        int64_t wake_at = 0;
        while (!srv->pending.empty()) {
            Request &head = srv->reqs[srv->pending.front()];
            if (head.not_before > now_ns()) {
                wake_at = head.not_before;
                break;
            }
            int slot = -1;
            for (size_t i = 0; i < srv->slots.size(); ++i)
                if (!srv->slot_busy[i]) {
                    slot = (int)i;
                    break;
                }
            if (slot < 0) break;
            size_t off = 0;
            if (!srv->arena.alloc(head.need, &off)) break;
            srv->pending.pop_front();
            head.off = off;
            head.slot = slot;
            head.t_start = now_ns();
            srv->slot_busy[slot] = 1;
            Request r = head;   // a copy: the map may change while unlocked
            int inject = EXSUM_OK;
            if (srv->fail_next > 0) {
                srv->fail_next--;
                inject = srv->fail_status;
            }
            lock.unlock();
            const int rc = inject != EXSUM_OK ? inject : launch(srv, r);
            int rc2 = EXSUM_OK;
            if (rc) {
                // Whatever was queued before the failure may still run: let
                // the stream release the request's memory and slot once it
                // drains.
                cudaGetLastError();
                Completion *c = new Completion{srv, r.ticket, rc};
                if (cudaLaunchHostFunc(srv->slots[slot], on_complete, c) != cudaSuccess) {
                    delete c;
                    cudaGetLastError();
                    rc2 = EXSUM_ECUDA;
                }
            }
            lock.lock();
            if (rc && rc2) {
                // No callback could be queued, so none will complete the
                // request: do it here.  Its arena block stays reserved until
                // the server is destroyed (work queued before the failure
                // may still use it).  When the callback was queued, it sets
                // the status together with `done`; the request may even be
                // released already, so it is not looked up here.
                auto it = srv->reqs.find(r.ticket);
                if (it != srv->reqs.end()) {
                    it->second.status = rc;
                    it->second.done = true;
                    it->second.t_done = now_ns();
                    srv->completed++;
                }
                srv->slot_busy[slot] = 0;
                srv->cv_done.notify_all();
            }
        }
        if (srv->stop && srv->pending.empty()) break;
        if (wake_at) {
            const int64_t dt = wake_at - now_ns();
            if (dt > 0) srv->cv_work.wait_for(lock, std::chrono::nanoseconds(dt));
        } else {
            srv->cv_work.wait_for(lock, std::chrono::milliseconds(5));
        }
    }
}

}  // namespace

extern "C" {

exsum_server *exsum_server_create(size_t mem_budget_bytes, int max_slots)
{
    if (mem_budget_bytes < 256 || max_slots < 1 || max_slots > 256) return nullptr;
    exsum_server *srv = new exsum_server();
    if (cudaGetDevice(&srv->device) != cudaSuccess) {
        delete srv;
        return nullptr;
    }
    if (cudaMalloc(&srv->arena_base, mem_budget_bytes) != cudaSuccess) {
        cudaGetLastError();
        delete srv;
        return nullptr;
    }
    srv->budget = mem_budget_bytes;
    srv->arena.reset(mem_budget_bytes);
    srv->slots.assign(max_slots, nullptr);
    srv->slot_busy.assign(max_slots, 0);
    for (int i = 0; i < max_slots; ++i) {
        if (cudaStreamCreateWithFlags(&srv->slots[i], cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (cudaStream_t s : srv->slots)
                if (s) cudaStreamDestroy(s);
            cudaFree(srv->arena_base);
            delete srv;
            return nullptr;
        }
        exsum::aux_prepare(srv->slots[i]);
    }
    srv->worker = std::thread(worker_main, srv);
    return srv;
}

int exsum_server_submit_at(exsum_server *srv, const exsum_desc *desc, int flags,
                           int64_t arrival_ns, uint64_t *ticket);

int exsum_server_submit(exsum_server *srv, const exsum_desc *desc, int flags, uint64_t *ticket)
{
    return exsum_server_submit_at(srv, desc, flags, 0, ticket);
}

int exsum_server_submit_at(exsum_server *srv, const exsum_desc *desc, int flags,
                           int64_t arrival_ns, uint64_t *ticket)
{
    if (!srv || !desc || !ticket) return EXSUM_EINVAL;
    if (flags & ~EXSUM_SERVE_HOST) return EXSUM_EINVAL;
    int st = 0;
    const size_t ws = exsum_workspace_bytes(desc->d, desc->shape, desc->k, desc->op, desc->dtype, 1,
                                            &st);
    if (st) return st;
    if (!desc->in || !desc->out) return EXSUM_EINVAL;
    Request r;
    r.desc = *desc;
    r.flags = flags;
    r.ws_bytes = ws;
    int64_t n = 1;
    for (int i = 0; i < desc->d; ++i) n *= desc->shape[i];
    if (flags & EXSUM_SERVE_HOST) {
        r.in_bytes = (size_t)n * exsum_dtype_size(desc->dtype);
        r.out_bytes = (size_t)n * exsum_dtype_size(exsum_out_dtype(desc->dtype));
    }
    r.need = ((ws + 255) & ~(size_t)255) + ((r.in_bytes + 255) & ~(size_t)255) +
             ((r.out_bytes + 255) & ~(size_t)255);
    if (r.need == 0) r.need = 256;
    if (r.need > srv->budget) return EXSUM_ENOMEM;   // could never be admitted
    r.t_submit = arrival_ns > 0 ? arrival_ns : now_ns();
    r.not_before = arrival_ns;
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        if (srv->stop) return EXSUM_EBUSY;
        r.ticket = srv->next_ticket++;
        *ticket = r.ticket;
        srv->reqs[r.ticket] = r;
        srv->pending.push_back(r.ticket);
    }
    srv->cv_work.notify_one();
    return EXSUM_OK;
}

int exsum_server_wait(exsum_server *srv, uint64_t ticket, int64_t timeout_ns)
{
    if (!srv) return EXSUM_EINVAL;
    std::unique_lock<std::mutex> lock(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return EXSUM_EINVAL;
    const auto deadline = std::chrono::steady_clock::now() +
                          std::chrono::nanoseconds(timeout_ns < 0 ? 0 : timeout_ns);
    // Looked up again after every wake: another thread may release the
    // ticket while this one waits.
    while (true) {
        it = srv->reqs.find(ticket);
        if (it == srv->reqs.end()) return EXSUM_EINVAL;
        if (it->second.done) return it->second.status;
        if (srv->cv_done.wait_until(lock, deadline) == std::cv_status::timeout) {
            it = srv->reqs.find(ticket);
            if (it == srv->reqs.end()) return EXSUM_EINVAL;
            return it->second.done ? it->second.status : EXSUM_ETIMEDOUT;
        }
    }
}

int exsum_server_ticket_times(exsum_server *srv, uint64_t ticket, int64_t *submit_ns,
                              int64_t *start_ns, int64_t *done_ns)
{
    if (!srv) return EXSUM_EINVAL;
    std::lock_guard<std::mutex> lock(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return EXSUM_EINVAL;
    if (!it->second.done) return EXSUM_EBUSY;
    if (submit_ns) *submit_ns = it->second.t_submit;
    if (start_ns) *start_ns = it->second.t_start;
    if (done_ns) *done_ns = it->second.t_done;
    return EXSUM_OK;
}

int exsum_server_release(exsum_server *srv, uint64_t ticket)
{
    if (!srv) return EXSUM_EINVAL;
    std::lock_guard<std::mutex> lock(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return EXSUM_EINVAL;
    if (!it->second.done) return EXSUM_EBUSY;
    srv->reqs.erase(it);
    return EXSUM_OK;
}

int64_t exsum_server_now_ns(void) { return now_ns(); }

int exsum_server_fail_next(exsum_server *srv, int count, int status)
{
    if (!srv || count < 0 || status >= 0) return EXSUM_EINVAL;
    std::lock_guard<std::mutex> lock(srv->mu);
    srv->fail_next = count;
    srv->fail_status = status;
    return EXSUM_OK;
}

int64_t exsum_server_completed(exsum_server *srv)
{
    if (!srv) return -1;
    std::lock_guard<std::mutex> lock(srv->mu);
    return srv->completed;
}

void exsum_server_destroy(exsum_server *srv)
{
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_one();
    if (srv->worker.joinable()) srv->worker.join();
    for (cudaStream_t s : srv->slots) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    cudaFree(srv->arena_base);
    delete srv;
}

}  // extern "C"
