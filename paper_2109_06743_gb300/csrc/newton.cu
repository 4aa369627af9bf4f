// Dispatch of the Newton fit kernels (newton.cuh) over the compiled
// velocity-block sizes; each size is instantiated in its own translation
// unit (newton_<N>.cu) so that the build compiles them in parallel.
#include "kernels.cuh"

namespace vl {

cudaError_t launch_newton_8(const FitArgs& a, cudaStream_t st);
cudaError_t launch_newton_12(const FitArgs& a, cudaStream_t st);
cudaError_t launch_newton_16(const FitArgs& a, cudaStream_t st);
cudaError_t launch_newton_20(const FitArgs& a, cudaStream_t st);
cudaError_t launch_newton_24(const FitArgs& a, cudaStream_t st);

cudaError_t launch_newton3d(const FitArgs& a, cudaStream_t st) {
    switch (a.nv) {
        case 8: return launch_newton_8(a, st);
        case 12: return launch_newton_12(a, st);
        case 16: return launch_newton_16(a, st);
        case 20: return launch_newton_20(a, st);
        case 24: return launch_newton_24(a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace vl
