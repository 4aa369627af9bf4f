// Measured arithmetic peak of the GPU (vl_fma_peak, include/vlasov.h): the
// denominator of the Newton fit's ALU roofline. The paper has no
// counterpart; it measures the machine, not the method.
//
// A kernel of independent fused multiply-add chains (eight per thread, so
// that the pipe, not the chains' latency, is the limit) over a grid of
// eight 256-thread blocks per SM, timed with CUDA events on the caller's
// stream after one untimed launch. The chains x <- x a + b with a < 1
// converge to b / (1 - a), so the values stay finite; the sum is compared
// with a value it never takes, so the compiler keeps every operation. No
// clock, power or other device setting is read or changed.
#include "common.cuh"
#include "kernels.cuh"

namespace vl {

template <typename T>
__global__ void __launch_bounds__(256) fma_chains_kernel(T* sink, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = T(threadIdx.x + k) * T(1e-3);
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == T(-1.25)) sink[0] = s;  // never true: keeps the chains alive
}

cudaError_t fma_peak(int precision, double* ops_per_s, void* sink, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)(8 * (sms > 0 ? sms : 1));
    const int iters = precision == 64 ? 256 : 32768;
    cudaEvent_t t0, t1;
    e = cudaEventCreate(&t0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&t1);
    if (e != cudaSuccess) {
        cudaEventDestroy(t0);
        return e;
    }
    float ms = 0.f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(t0, st);
        if (e != cudaSuccess) break;
        if (precision == 64)
            fma_chains_kernel<double><<<grid, 256, 0, st>>>(static_cast<double*>(sink), iters, 0.9999, 1e-4);
        else
            fma_chains_kernel<float><<<grid, 256, 0, st>>>(static_cast<float*>(sink), iters, 0.9999f, 1e-4f);
        count_launch();
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(t1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (e != cudaSuccess) return e;
    const double fmas = (double)grid * 256.0 * (double)iters * 16.0 * 8.0;
    *ops_per_s = ms > 0.f ? fmas / (ms * 1e-3) : 0.0;
    return cudaSuccess;
}

}  // namespace vl
