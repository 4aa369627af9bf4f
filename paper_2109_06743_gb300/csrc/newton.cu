// Dispatch of the 2D3V Newton fit kernels over the compiled velocity-block
// sizes and the two arithmetics (newton.cuh: double-float on the FP32 pipe;
// newton64.cuh: plain FP64); each size is instantiated in its own
// translation unit (newton_<N>.cu) so that the build compiles them in
// parallel. Also the device-side choice between the two double-float
// kernels (fit_select_kernel).
#include "kernels.cuh"

namespace vl {

cudaError_t launch_newton_8(const FitArgs& a, cudaStream_t st);
cudaError_t launch_newton_12(const FitArgs& a, cudaStream_t st);
cudaError_t launch_newton_16(const FitArgs& a, cudaStream_t st);
cudaError_t launch_newton_20(const FitArgs& a, cudaStream_t st);
cudaError_t launch_newton_24(const FitArgs& a, cudaStream_t st);
cudaError_t launch_newton64_8(const FitArgs& a, cudaStream_t st);
cudaError_t launch_newton64_12(const FitArgs& a, cudaStream_t st);
cudaError_t launch_newton64_16(const FitArgs& a, cudaStream_t st);
cudaError_t launch_newton64_20(const FitArgs& a, cudaStream_t st);
cudaError_t launch_newton64_24(const FitArgs& a, cudaStream_t st);

cudaError_t launch_newton3d(const FitArgs& a, cudaStream_t st) {
    if (a.fp64) {
        switch (a.nv) {
            case 8: return launch_newton64_8(a, st);
            case 12: return launch_newton64_12(a, st);
            case 16: return launch_newton64_16(a, st);
            case 20: return launch_newton64_20(a, st);
            case 24: return launch_newton64_24(a, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (a.nv) {
        case 8: return launch_newton_8(a, st);
        case 12: return launch_newton_12(a, st);
        case 16: return launch_newton_16(a, st);
        case 20: return launch_newton_20(a, st);
        case 24: return launch_newton_24(a, st);
        default: return cudaErrorInvalidValue;
    }
}

// Decrease of the exponent of the Maxwellian with targets t from its peak to
// the farthest corner of the velocity box, summed over the axes from the
// diagonal of Theta (a cell's values span about this many e-folds). Empty
// or invalid targets give 0.
__device__ double box_spread(const double* t, const double* vmin, const double* vmax) {
    const double n = t[0];
    if (!(n > 0.0) || !isfinite(n)) return 0.0;
    const int diag[3] = {4, 7, 9};
    double s = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double u = t[1 + a] / n;
        const double th = fmax(t[diag[a]] / n - u * u, 1e-300);
        const double ext = fmax(vmax[a] - u, u - vmin[a]);
        s += ext * ext / (2.0 * th);
    }
    return isfinite(s) ? s : 0.0;
}

// One thread per cell: the largest n over all cells (sel[0]) and over the
// cells whose V (moments of f) or F (fluid) Maxwellian spans more than 60
// e-folds over the box (sel[1]), as FP64 bit patterns (positive doubles
// order like their bits). The double-float fit's common evaluation needs
// every value of a block within e^+-80 and the peak itself lies some
// e-folds below 1; cells below 1e-10 of the largest density (whose fits do
// not matter) do not choose the kernel.
__global__ void fit_select_kernel(FitArgs a, unsigned long long* sel) {
    unsigned long long top = 0ull, wide = 0ull;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < a.ncell;
         c += (long long)gridDim.x * blockDim.x) {
        double tv[10], tf[10];
        for (int q = 0; q < 10; ++q) {
            tv[q] = a.vmom[c * 20 + q];
            tf[q] = a.fluid[c * 10 + q];
        }
        const double n = tv[0];
        if (!(n > 0.0) || !isfinite(n)) continue;
        const unsigned long long bits = (unsigned long long)__double_as_longlong(n);
        top = max(top, bits);
        if (fmax(box_spread(tv, a.vmin, a.vmax), box_spread(tf, a.vmin, a.vmax)) > 60.0) wide = max(wide, bits);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        top = max(top, __shfl_xor_sync(0xffffffffu, top, o));
        wide = max(wide, __shfl_xor_sync(0xffffffffu, wide, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (top) atomicMax(&sel[0], top);
        if (wide) atomicMax(&sel[1], wide);
    }
}

cudaError_t launch_fit_select(const FitArgs& a, unsigned long long* sel, cudaStream_t st) {
    long long blocks = (a.ncell + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    fit_select_kernel<<<(unsigned)blocks, 256, 0, st>>>(a, sel);
    count_launch();
    return cudaGetLastError();
}

}  // namespace vl
