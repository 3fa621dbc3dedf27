// kernels_longrow.cuh -- the final pass of the row schedule for rows longer
// than one warp can scan (over 1024 elements): one block per row.
//
// Same result as k_rowx without the window along n_{d-1} (that window is a
// strided pass of its own for such rows): for every row x' of the input H
// (the BDBS of the tensor along dimensions 1..d-1) and every x_d,
//
//   out[x', x_d] = T[x'] (+) (+)_{y < x_d} H[x', y] (+) (+)_{y >= x_d + k_d} H[x', y]
//
// (Sec. 4: the regions of the excluded-sum components along dimension d,
// plus the lower-dimensional part T).  Thread t of the block owns the strip
// of V consecutive elements from t V.  Within a strip the exclusive prefixes
// and inclusive suffixes are taken in the local type; across strips the
// strip totals are scanned in both directions in the long (compensated)
// accumulator, by warp shuffles and then the warp totals (a fixed order).
// The strips' local suffixes go to shared memory, with each strip's suffix
// of the strips after it, so that an output reads the suffix from x_d + k_d
// (in any strip) back: its long part is T (+) the prefix before its strip
// (+) the suffix after the strip of x_d + k_d -- at most two values per
// thread -- and its local part the in-strip prefix (+) the in-strip suffix.
#pragma once

#include "kernels_line1d.cuh"

namespace exsum {

template <class M, class SIn, class SOut, int NT, int V>
__global__ void __launch_bounds__(NT)
k_rowx_long(const SIn *__restrict__ H, const typename M::car_t *__restrict__ T, SOut *__restrict__ out,
            int64_t rows, int L, int k3)
{
    using Lt = typename M::loc_t;
    using A = typename M::acc_t;
    extern __shared__ __align__(16) unsigned char lr_smem[];
    Lt *Ssh = reinterpret_cast<Lt *>(lr_smem);                                   // local suffixes, L
    A *Aft = reinterpret_cast<A *>(lr_smem + (((size_t)NT * V * sizeof(Lt) + 15) & ~(size_t)15));  // per strip
    const int tid = threadIdx.x;
    const int s0 = tid * V;
    constexpr int LV = V == 4 ? 2 : V == 8 ? 3 : V == 16 ? 4 : 5;
    const uint64_t pol_in = l2_policy_evict_first();
    const uint64_t pol_out = l2_policy_evict_first();
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const SIn *h = H + row * (int64_t)L;
        SOut *o = out + row * (int64_t)L;
        const int valid = max(0, min(V, L - s0));
        Lt v[V];
        load_strip<M, SIn, V>(h + (valid > 0 ? s0 : 0), ((uintptr_t)(h + s0) & 15) == 0, valid, v, pol_in);
        // in-strip exclusive prefixes (in place) and inclusive suffixes
        Lt s[V];
        s[V - 1] = v[V - 1];
#pragma unroll
        for (int j = V - 2; j >= 0; --j) s[j] = M::lop(v[j], s[j + 1]);
        Lt run = M::lid();
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const Lt x = v[j];
            v[j] = run;
            run = M::lop(run, x);
        }
        A pre, suf;
        block_exscan_pair<M, NT, true>(run, s[0], pre, suf);
        if (valid > 0) {
#pragma unroll
            for (int j = 0; j < V; ++j)
                if (j < valid) Ssh[s0 + j] = s[j];
        }
        Aft[tid] = suf;
        __syncthreads();
        if (valid > 0) {
            // long parts for the (at most two) strips the suffix reads fall in
            const A tv = M::get(T[row]);
            const A tp = M::op(tv, pre);
            const int sy = (s0 + k3) >> LV;
            const A l0 = sy < NT ? M::op(tp, Aft[sy]) : tp;
            const A l1 = sy + 1 < NT ? M::op(tp, Aft[sy + 1]) : tp;
            SOut res[V];
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const int y = s0 + j + k3;
                if (y < L)
                    res[j] = finish<M, SOut>((y >> LV) == sy ? l0 : l1, M::lop(v[j], Ssh[y]));
                else
                    res[j] = finish<M, SOut>(tp, v[j]);
            }
            if (sizeof(SOut) == 4 && valid == V && ((uintptr_t)(o + s0) & 15) == 0) {
#pragma unroll
                for (int i = 0; i < V / 4; ++i) {
                    uint4 w;
                    memcpy(&w, res + 4 * i, 16);
                    st_hint_v4(o + s0 + 4 * i, w, pol_out);
                }
            } else {
#pragma unroll
                for (int j = 0; j < V; ++j)
                    if (j < valid) st_hint(o + s0 + j, res[j], pol_out);
            }
        }
        __syncthreads();   // Ssh and Aft are rewritten for the next row
    }
}

// Shared memory of k_rowx_long: the local suffixes of a row and one long
// value per strip.
template <class M>
inline size_t rowx_long_smem(int nt, int v)
{
    return (((size_t)nt * v * sizeof(typename M::loc_t) + 15) & ~(size_t)15) + (size_t)nt * sizeof(typename M::acc_t);
}

}  // namespace exsum
