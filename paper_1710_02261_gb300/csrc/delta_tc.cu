// delta_tc.cu -- Eq. (delta) on tcgen05 tensor cores (filled in below).
#include "common.cuh"

namespace ptk {

bool delta_tc_supported(const DeltaJob&, ptk_precision) { return false; }

ptk_status delta_tc(ptk_ctx*, const DeltaJob&, ptk_precision, cudaStream_t) {
    set_error("tensor-core delta is not available for this shape");
    return PTK_ERR_UNSUPPORTED;
}

}  // namespace ptk
