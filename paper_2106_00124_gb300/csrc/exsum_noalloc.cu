// exsum_noalloc.cu -- excluded sums for callers that cannot allocate device
// memory at call time.
//
// Some callers have no way to call cudaMalloc when they need an excluded sum:
// a plugin living inside a host framework that owns the whole device-memory
// budget through its own allocator, a real-time loop that cannot afford the
// implicit device synchronisation of cudaMalloc/cudaFree, or an embedded
// deployment whose allocations are all fixed at start-up.  For them this
// file provides exsum_excluded_noalloc(), which runs the same excluded-sum
// pipeline as exsum_excluded_ws() on a fixed scratch buffer that is part of
// the library image: a file-scope __device__ array of
// EXSUM_NOALLOC_SCRATCH_BYTES bytes.  Every GPU that loads the library holds
// that buffer until the process exits.
//
// The array's name, used in host code, is only a host-side stand-in for the
// device variable; passing it to a kernel would fault or (where the GPU can
// reach host memory) silently use the wrong memory.  The device address is
// therefore looked up with cudaGetSymbolAddress, with the device current, on
// the first call made on that device and again on every later call made
// outside a stream capture (a device reset moves it).
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/exsum.h"

static __device__ __align__(256) unsigned char g_noalloc_scratch[EXSUM_NOALLOC_SCRATCH_BYTES];

namespace exsum {
int excluded_ws_serial(const void *in, void *out, int d, const int64_t *shape, const int64_t *k,
                       int op, int dtype, void *workspace, size_t workspace_bytes, void *stream);
}

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};
}  // namespace

extern "C" int exsum_excluded_noalloc(const void *in, void *out, int d, const int64_t *shape,
                                      const int64_t *k, int op, int dtype, void *stream)
{
    int status = EXSUM_OK;
    const size_t need = exsum_workspace_bytes(d, shape, k, op, dtype, 1, &status);
    if (status != EXSUM_OK) return status;
    if (!in || !out) return EXSUM_EINVAL;
    if (need > (size_t)EXSUM_NOALLOC_SCRATCH_BYTES) return EXSUM_ENOMEM;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return EXSUM_ECUDA;
    // The address is looked up again on every call made outside a stream
    // capture, so that a device reset (which reloads the library's device
    // image at a new address) never leaves a stale pointer behind; inside a
    // capture the address from the last uncaptured call is used.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess) {
        cudaGetLastError();
        return EXSUM_ECUDA;
    }
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (cs == cudaStreamCaptureStatusNone || !g_noalloc_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return EXSUM_ECUDA;
            }
            g_noalloc_ptr[dev] = p;
        }
        scratch = g_noalloc_ptr[dev];
    }
    // Serial schedule: no side stream or event is created on this path.
    return exsum::excluded_ws_serial(in, out, d, shape, k, op, dtype, scratch,
                                     (size_t)EXSUM_NOALLOC_SCRATCH_BYTES, stream);
}
