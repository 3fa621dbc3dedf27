// exsum_cmp.cu -- C ABI of the paper's comparison methods on the GPU
// (kernels_cmp.cuh): summed-area tables with inclusion-exclusion for
// integer + (Sec. 1), and the corners algorithm for d = 2 and 3 (App. A).
// Both run on the caller's stream with the library's cached workspace.
#include "cmp_run.cuh"

namespace {
using namespace exsum;
using namespace exsum::cmp;
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
