// Newton fit kernels for 24^3 velocity blocks: double-float (newton.cuh)
// and FP64 (newton64.cuh).
#include "newton.cuh"
#include "newton64.cuh"

namespace vl {
cudaError_t launch_newton_24(const FitArgs& a, cudaStream_t st) { return launch_n<24>(a, st); }
cudaError_t launch_newton64_24(const FitArgs& a, cudaStream_t st) { return fit64::launch64<24>(a, st); }
}  // namespace vl
