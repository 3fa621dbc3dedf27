// cmp_run.cuh -- host side of the comparison methods (kernels_cmp.cuh):
// scan plans, and the SAT and corners pipelines on one stream, templated on
// the monoid.  Included by exsum_cmp.cu and exsum_slow.cu.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/exsum.h"
#include "kernels_cmp.cuh"

namespace exsum {
int cached_ws(void *stream, size_t need, void **ws, size_t *bytes);                    // exsum_abi.cu
int validate_args(int d, const int64_t *shape, const int64_t *k, int op, int dtype);   // exsum_abi.cu

namespace cmp {

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

inline int64_t volume(int d, const int64_t *n)
{
    int64_t v = 1;
    for (int i = 0; i < d; ++i) v *= n[i];
    return v;
}

inline CmpDims dims_of(int d, const int64_t *n, const int64_t *k)
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

// Segments of a scan along dimension j: none (G = n) when the lines alone
// give the GPU enough threads (warps for the contiguous dimension), else
// about 256K threads (16K warps) over the line segments.
struct ScanPlan {
    int64_t O, I, G, nseg;
};

inline ScanPlan scan_plan(int d, const int64_t *n, int j)
{
    ScanPlan p{1, 1, n[j], 1};
    for (int i = 0; i < j; ++i) p.O *= n[i];
    for (int i = j + 1; i < d; ++i) p.I *= n[i];
    const int64_t lines = p.O * p.I;
    const int64_t want = p.I == 1 ? 16384 : 262144;   // warps / threads
    if (lines < want) {
        const int64_t minlen = p.I == 1 ? 1024 : 64;
        const int64_t nseg = std::min(cdiv(n[j], minlen), cdiv(want, lines));
        if (nseg > 1) {
            p.G = cdiv(n[j], nseg);
            p.nseg = cdiv(n[j], p.G);
        }
    }
    return p;
}

// Carry elements the segmented scans of a tensor need, over all dimensions.
inline int64_t scan_carry_elems(int d, const int64_t *n)
{
    int64_t m = 0;
    for (int j = 0; j < d; ++j) {
        const ScanPlan p = scan_plan(d, n, j);
        if (p.nseg > 1) m = std::max(m, p.O * p.nseg * p.I);
    }
    return m;
}

// Inclusive prefix (or suffix) along dimension j of the tensor `in` into
// `out` (`in` may be `out`); Cy: carries of a segmented scan.
template <class M, class SR, class SW, bool SUF>
void scan_dim_t(const SR *in, SW *out, SW *Cy, int d, const int64_t *n, int j, cudaStream_t s)
{
    const ScanPlan p = scan_plan(d, n, j);
    if (p.nseg > 1) {
        const int64_t units = p.I == 1 ? p.O * p.nseg * 32 : p.O * p.nseg * p.I;
        k_scan_seg<M, SR, SW, SUF><<<(unsigned)cdiv(units, 256), 256, 0, s>>>(in, out, p.O, n[j], p.I, p.G, p.nseg);
        k_seg_carry<M, SW, SUF><<<(unsigned)cdiv(p.O * p.I * 32, 256), 256, 0, s>>>(out, Cy, p.O, n[j], p.I, p.G, p.nseg);
        k_seg_apply<M, SW, SUF><<<(unsigned)cdiv(p.O * n[j] * p.I, 256), 256, 0, s>>>(out, Cy, p.O, n[j], p.I,
                                                                                      p.G, p.nseg);
    } else if (p.I == 1) {
        k_scan_rows<M, SR, SW, SUF><<<(unsigned)cdiv(p.O * 32, 256), 256, 0, s>>>(in, out, p.O, n[j]);
    } else {
        k_scan_lines<M, SR, SW, SUF><<<(unsigned)cdiv(p.O * p.I, 256), 256, 0, s>>>(in, out, p.O, n[j], p.I);
    }
}

template <class M, class SR, class SW>
void scan_dim(const SR *in, SW *out, SW *Cy, int d, const int64_t *n, int j, bool suffix, cudaStream_t s)
{
    if (suffix)
        scan_dim_t<M, SR, SW, true>(in, out, Cy, d, n, j, s);
    else
        scan_dim_t<M, SR, SW, false>(in, out, Cy, d, n, j, s);
}

inline int finish(cudaStream_t s)
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
    const size_t sb = ((size_t)N * sizeof(T) + 255) & ~(size_t)255;
    void *ws = nullptr;
    size_t wsb = 0;
    int rc = cached_ws(stream, sb + (size_t)scan_carry_elems(d, n) * sizeof(T), &ws, &wsb);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    T *S = static_cast<T *>(ws);
    T *Cy = reinterpret_cast<T *>(static_cast<char *>(ws) + sb);
    // the summed-area table: the prefix along every dimension (in place after the first)
    scan_dim<M, T, T>(static_cast<const T *>(in), S, Cy, d, n, 0, false, s);
    for (int j = 1; j < d; ++j) scan_dim<M, T, T>(S, S, Cy, d, n, j, false, s);
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
    int rc = cached_ws(stream, one * (size_t)tensors + (size_t)scan_carry_elems(d, n) * sizeof(C), &ws, &wsb);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    char *base = static_cast<char *>(ws);
    C *Cy = reinterpret_cast<C *>(base + one * (size_t)tensors);
    C *lvl[3][8] = {};
    int64_t used = 0;
    for (int j = 0; j < d; ++j)
        for (int b = 0; b < (2 << j); ++b) lvl[j][b] = reinterpret_cast<C *>(base + one * (size_t)used++);
    // level 0 from the input; tensor b of level j: bit i set = suffix along dimension i
    scan_dim<M, IN, C>(static_cast<const IN *>(in), lvl[0][0], Cy, d, n, 0, false, s);
    scan_dim<M, IN, C>(static_cast<const IN *>(in), lvl[0][1], Cy, d, n, 0, true, s);
    for (int j = 1; j < d; ++j)
        for (int b = 0; b < (2 << j); ++b)
            scan_dim<M, C, C>(lvl[j - 1][b & ((1 << j) - 1)], lvl[j][b], Cy, d, n, j, (b >> j) & 1, s);
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

}  // namespace cmp
}  // namespace exsum
