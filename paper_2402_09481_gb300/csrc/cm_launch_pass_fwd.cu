// Forward column passes over the Goldilocks field.
#include "cm_launch_pass.cuh"

namespace cm {
cudaError_t launch_pass_fwd(const PassArgs &a, int logr, cudaStream_t st) {
    return launch_pass_dispatch<FieldGL, false>(a, logr, st);
}
}  // namespace cm
