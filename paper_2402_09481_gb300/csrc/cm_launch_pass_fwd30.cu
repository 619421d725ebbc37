// Forward column passes over the field of 3 * 2^30 + 1.
#include "cm_launch_pass.cuh"

namespace cm {
cudaError_t launch_pass_fwd30(const PassArgs &a, int logr, cudaStream_t st) {
    return launch_pass_dispatch<FieldF30, false>(a, logr, st);
}
}  // namespace cm
