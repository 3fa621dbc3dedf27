// exsum_slow.cu -- the cost of the operator, measured (the paper's
// experiment with an artificially slowed (+), Sec. 6): int64 + whose every
// application also runs a chain of `extra` dependent steps that leave its
// value unchanged (set at run time), through the same pipelines as the library's own calls --
// box-complement's row schedule, BDBS and corners -- plus a calibration
// kernel that applies the operator a known number of times per element.
// Once the extra work dominates, time grows linearly with `extra`, and the
// ratio of a method's slope to the calibration's slope per application is
// the number of operator applications per element the method performs.
#include "cmp_run.cuh"
#include "pipeline.cuh"

namespace exsum {

// extra dependent steps per application of the slowed operator, and a zero
// the compiler cannot see (so that the steps are not folded away)
__device__ int g_slow_extra;
__device__ uint64_t g_slow_zero;

struct MonSlowAdd : MonIntAdd<int64_t, uint64_t> {
    __device__ __forceinline__ static int64_t op(int64_t a, int64_t b)
    {
        uint64_t s = (uint64_t)a + (uint64_t)b;
        const int n = g_slow_extra;
        const uint64_t z = g_slow_zero;
        for (int i = 0; i < n; ++i) s = (s ^ z) + z;   // s unchanged, one dependent step
        return (int64_t)s;
    }
    __device__ __forceinline__ static int64_t lop(int64_t a, int64_t b) { return op(a, b); }
};

// Calibration: every element folds its input into itself `reps` times (reps
// applications per element), with one read and one write.
__global__ void __launch_bounds__(256) k_slow_calib(const int64_t *__restrict__ in, int64_t *__restrict__ out,
                                                    int64_t N, int reps)
{
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= N) return;
    const int64_t x = in[gid];
    int64_t acc = x;
    for (int r = 0; r < reps; ++r) acc = MonSlowAdd::op(acc, x);
    out[gid] = acc;
}

}  // namespace exsum

namespace {
using namespace exsum;
using namespace exsum::cmp;

int pipe_run(int excluded, const void *in, void *out, int d, const int64_t *n, const int64_t *k, void *stream)
{
    size_t need = 0;
    cudaError_t err = cudaSuccess;
    int rc = Pipe<MonSlowAdd>::run(excluded, nullptr, nullptr, d, n, k, nullptr, 0, (cudaStream_t)stream, &need,
                                   &err, nullptr);
    if (rc) return rc;
    void *ws = nullptr;
    size_t wsb = 0;
    rc = cached_ws(stream, need, &ws, &wsb);
    if (rc) return rc;
    rc = Pipe<MonSlowAdd>::run(excluded, in, out, d, n, k, ws, wsb, (cudaStream_t)stream, nullptr, &err, nullptr);
    return rc;
}
}  // namespace

extern "C" {

int exsum_slow_extra(int extra)
{
    if (extra < 0) return EXSUM_EINVAL;
    const uint64_t zero = 0;
    cudaError_t e = cudaMemcpyToSymbol(g_slow_extra, &extra, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_slow_zero, &zero, sizeof(zero));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return EXSUM_ECUDA;
    }
    return EXSUM_OK;
}

int exsum_slow_run(const void *in, void *out, int d, const int64_t *shape, const int64_t *k, int method,
                   void *stream)
{
    int rc = validate_args(d, shape, k, EXSUM_OP_ADD, EXSUM_I64);
    if (rc) return rc;
    if (!in || !out) return EXSUM_EINVAL;
    switch (method) {
    case EXSUM_SLOW_BOX_COMPLEMENT: return pipe_run(1, in, out, d, shape, k, stream);
    case EXSUM_SLOW_BDBS: return pipe_run(0, in, out, d, shape, k, stream);
    case EXSUM_SLOW_CORNERS:
        if (d != 2 && d != 3) return EXSUM_EUNSUPPORTED;
        return corners_run<MonSlowAdd>(in, out, d, shape, k, stream);
    case EXSUM_SLOW_CALIBRATE: {
        const int64_t N = cmp::volume(d, shape);
        k_slow_calib<<<(unsigned)cmp::cdiv(N, 256), 256, 0, (cudaStream_t)stream>>>(
            static_cast<const int64_t *>(in), static_cast<int64_t *>(out), N, EXSUM_SLOW_CALIBRATE_REPS);
        return finish((cudaStream_t)stream);
    }
    default: return EXSUM_EINVAL;
    }
}

}  // extern "C"
