// Newton fit kernel for 12^3 velocity blocks (see newton.cuh).
#include "newton.cuh"

namespace vl {
cudaError_t launch_newton_12(const FitArgs& a, cudaStream_t st) { return launch_n<12>(a, st); }
}  // namespace vl
