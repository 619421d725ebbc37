// Inverse column passes over the Goldilocks field.
#include "cm_launch_pass.cuh"

namespace cm {
cudaError_t launch_pass_inv(const PassArgs &a, int logr, cudaStream_t st) {
    return launch_pass_dispatch<FieldGL, true>(a, logr, st);
}
}  // namespace cm
