// Newton fit kernel for 8^3 velocity blocks (see newton.cuh).
#include "newton.cuh"

namespace vl {
cudaError_t launch_newton_8(const FitArgs& a, cudaStream_t st) { return launch_n<8>(a, st); }
}  // namespace vl
