// Inverse column passes over the field of 5 * 2^25 + 1.
#include "cm_launch_pass.cuh"

namespace cm {
cudaError_t launch_pass_inv25(const PassArgs &a, int logr, cudaStream_t st) {
    return launch_pass_dispatch<FieldF25, true>(a, logr, st);
}
}  // namespace cm
