// Newton fit kernel for 24^3 velocity blocks (see newton.cuh).
#include "newton.cuh"

namespace vl {
cudaError_t launch_newton_24(const FitArgs& a, cudaStream_t st) { return launch_n<24>(a, st); }
}  // namespace vl
