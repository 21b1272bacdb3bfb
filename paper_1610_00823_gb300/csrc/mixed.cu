// Split-precision near-field operands (VFMM_MIXED).
#include "ops.cuh"
#include "vfmm_internal.cuh"

namespace vfmm {

int mixed_prepare(vfmm_ops* o, cudaStream_t st) {
    (void)o;
    (void)st;
    return fail(VFMM_ERR_INVALID_ARG, "VFMM_MIXED is not available in this build");
}

void mixed_free(vfmm_ops* o) { o->mixed = nullptr; }

}  // namespace vfmm
