// Instantiates the included/excluded pipelines for BF16 inputs (both operators).
#include "pipeline.cuh"

namespace exsum {

int dispatch_bf16(int op, int excluded, const void *in, void *out, int d, const int64_t *n,
                   const int64_t *k, void *ws, size_t ws_bytes, cudaStream_t stream,
                   size_t *ws_needed, cudaError_t *cuda_err, const Aux *aux)
{
    if (op == OP_ADD)
        return Pipe<M_BF16_ADD>::run(excluded, in, out, d, n, k, ws, ws_bytes, stream, ws_needed,
                                     cuda_err, aux);
    return Pipe<M_BF16_MAX>::run(excluded, in, out, d, n, k, ws, ws_bytes, stream, ws_needed,
                                 cuda_err, aux);
}

}  // namespace exsum
