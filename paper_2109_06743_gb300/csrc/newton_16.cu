// Newton fit kernel for 16^3 velocity blocks (see newton.cuh).
#include "newton.cuh"

namespace vl {
cudaError_t launch_newton_16(const FitArgs& a, cudaStream_t st) { return launch_n<16>(a, st); }
}  // namespace vl
