// exsum_cmp.cu -- C ABI of the paper's comparison methods on the GPU
// (kernels_cmp.cuh): summed-area tables with inclusion-exclusion for
// integer + (Sec. 1), and the corners algorithm for d = 2 and 3 (App. A).
// Both run on the caller's stream with the library's cached workspace.
#include <cuda_runtime.h>

#include "../../include/exsum.h"
#include "kernels_cmp.cuh"

namespace exsum {
int cached_ws(void *stream, size_t need, void **ws, size_t *bytes);                    // exsum_abi.cu
int validate_args(int d, const int64_t *shape, const int64_t *k, int op, int dtype);   // exsum_abi.cu
}

namespace {

using namespace exsum;

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

int64_t volume(int d, const int64_t *n)
{
    int64_t v = 1;
    for (int i = 0; i < d; ++i) v *= n[i];
    return v;
}

CmpDims dims_of(int d, const int64_t *n, const int64_t *k)
{
    CmpDims g{};
    g.d = d;
    int64_t s = 1;
    for (int i = d - 1; i >= 0; --i) {
        g.n[i] = n[i];
        g.k[i] = k[i];
        g.st[i] = s;
        s *= n[i];
    }
    return g;
}

// Inclusive prefix (or suffix) along dimension j of the tensor `in` into `out`.
template <class M, class SR, class SW>
void scan_dim(const SR *in, SW *out, int d, const int64_t *n, int j, bool suffix, cudaStream_t s)
{
    int64_t O = 1, I = 1;
    for (int i = 0; i < j; ++i) O *= n[i];
    for (int i = j + 1; i < d; ++i) I *= n[i];
    if (I == 1) {
        const unsigned grid = (unsigned)cdiv(O * 32, 256);
        if (suffix)
            k_scan_rows<M, SR, SW, true><<<grid, 256, 0, s>>>(in, out, O, n[j]);
        else
            k_scan_rows<M, SR, SW, false><<<grid, 256, 0, s>>>(in, out, O, n[j]);
    } else {
        const unsigned grid = (unsigned)cdiv(O * I, 256);
        if (suffix)
            k_scan_lines<M, SR, SW, true><<<grid, 256, 0, s>>>(in, out, O, n[j], I);
        else
            k_scan_lines<M, SR, SW, false><<<grid, 256, 0, s>>>(in, out, O, n[j], I);
    }
}

int finish(cudaStream_t s)
{
    (void)s;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EXSUM_OK : EXSUM_ECUDA;
}

template <class T, class U>
int sat_run(const void *in, void *out, int d, const int64_t *n, const int64_t *k, int excluded, void *stream)
{
    using M = MonIntAdd<T, U>;
    const int64_t N = volume(d, n);
    void *ws = nullptr;
    size_t wsb = 0;
    int rc = cached_ws(stream, (size_t)N * sizeof(T), &ws, &wsb);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    T *S = static_cast<T *>(ws);
    // the summed-area table: the prefix along every dimension (in place after the first)
    scan_dim<M, T, T>(static_cast<const T *>(in), S, d, n, 0, false, s);
    for (int j = 1; j < d; ++j) scan_dim<M, T, T>(S, S, d, n, j, false, s);
    k_satc<T, U><<<(unsigned)cdiv(N, 256), 256, 0, s>>>(S, static_cast<T *>(out), dims_of(d, n, k), N, excluded);
    return finish(s);
}

template <class M>
int corners_run(const void *in, void *out, int d, const int64_t *n, const int64_t *k, void *stream)
{
    using IN = typename M::in_t;
    using C = typename M::car_t;
    using OUT = typename M::out_t;
    const int64_t N = volume(d, n);
    // the scan tree: level j holds the 2^(j+1) tensors of dimensions 0..j
    int64_t tensors = 0;
    for (int j = 0; j < d; ++j) tensors += (int64_t)2 << j;
    void *ws = nullptr;
    size_t wsb = 0;
    const size_t one = ((size_t)N * sizeof(C) + 255) & ~(size_t)255;
    int rc = cached_ws(stream, one * (size_t)tensors, &ws, &wsb);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    char *base = static_cast<char *>(ws);
    C *lvl[3][8] = {};
    int64_t used = 0;
    for (int j = 0; j < d; ++j)
        for (int b = 0; b < (2 << j); ++b) lvl[j][b] = reinterpret_cast<C *>(base + one * (size_t)used++);
    // level 0 from the input; tensor b of level j: bit i set = suffix along dimension i
    scan_dim<M, IN, C>(static_cast<const IN *>(in), lvl[0][0], d, n, 0, false, s);
    scan_dim<M, IN, C>(static_cast<const IN *>(in), lvl[0][1], d, n, 0, true, s);
    for (int j = 1; j < d; ++j)
        for (int b = 0; b < (2 << j); ++b)
            scan_dim<M, C, C>(lvl[j - 1][b & ((1 << j) - 1)], lvl[j][b], d, n, j, (b >> j) & 1, s);
    CornerTensors T{};
    for (int b = 0; b < (1 << d); ++b) T.t[b] = lvl[d - 1][b];
    const CmpDims g = dims_of(d, n, k);
    const unsigned grid = (unsigned)cdiv(N, 256);
    if (d == 2)
        k_corners<M, C, OUT, 2><<<grid, 256, 0, s>>>(T, static_cast<OUT *>(out), g, N);
    else
        k_corners<M, C, OUT, 3><<<grid, 256, 0, s>>>(T, static_cast<OUT *>(out), g, N);
    return finish(s);
}

}  // namespace

extern "C" {

int exsum_sat(const void *in, void *out, int d, const int64_t *shape, const int64_t *k, int excluded, int dtype,
              void *stream)
{
    int rc = validate_args(d, shape, k, EXSUM_OP_ADD, dtype);
    if (rc) return rc;
    if (!in || !out) return EXSUM_EINVAL;
    if (dtype == EXSUM_I32) return sat_run<int32_t, uint32_t>(in, out, d, shape, k, excluded != 0, stream);
    if (dtype == EXSUM_I64) return sat_run<int64_t, uint64_t>(in, out, d, shape, k, excluded != 0, stream);
    return EXSUM_EUNSUPPORTED;   // needs an inverse: integer + only
}

int exsum_corners(const void *in, void *out, int d, const int64_t *shape, const int64_t *k, int op, int dtype,
                  void *stream)
{
    int rc = validate_args(d, shape, k, op, dtype);
    if (rc) return rc;
    if (!in || !out) return EXSUM_EINVAL;
    if (d != 2 && d != 3) return EXSUM_EUNSUPPORTED;
    const bool add = op == EXSUM_OP_ADD;
    switch (dtype) {
    case EXSUM_I32: return add ? corners_run<M_I32_ADD>(in, out, d, shape, k, stream)
                               : corners_run<M_I32_MAX>(in, out, d, shape, k, stream);
    case EXSUM_I64: return add ? corners_run<M_I64_ADD>(in, out, d, shape, k, stream)
                               : corners_run<M_I64_MAX>(in, out, d, shape, k, stream);
    case EXSUM_F32: return add ? corners_run<M_F32_ADD>(in, out, d, shape, k, stream)
                               : corners_run<M_F32_MAX>(in, out, d, shape, k, stream);
    default: return add ? corners_run<M_BF16_ADD>(in, out, d, shape, k, stream)
                        : corners_run<M_BF16_MAX>(in, out, d, shape, k, stream);
    }
}

int exsum_corner_region(int d, int corner, int dim)
{
    if ((d != 2 && d != 3) || corner < 0 || corner >= (1 << d) || dim < 0 || dim >= d) return -1;
    return corner_region(d, corner, dim);
}

}  // extern "C"
