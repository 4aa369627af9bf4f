// Newton fit kernel for 20^3 velocity blocks (see newton.cuh).
#include "newton.cuh"

namespace vl {
cudaError_t launch_newton_20(const FitArgs& a, cudaStream_t st) { return launch_n<20>(a, st); }
}  // namespace vl
