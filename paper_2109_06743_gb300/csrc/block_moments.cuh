// Moments of a velocity block reduced over a CTA (paper Sec. 2.1: the 20 raw
// moments up to third order that feed the fluid step and the fit).
//
// Every thread owns one velocity line and forms its sums S_p = sum xi^p f
// (p = 0..3) in centred indices xi = index - (N-1)/2, which are exact in
// binary floating point; the 20 per-line products are reduced with warp
// shuffles in T and across warps in FP64 by lanes 0..19 of warp 0, which then
// expand them to physical velocities with the precomputed binomial table
// (MomConv, FP64).
#pragma once

#include "kernels.cuh"

namespace vl {

// moment order: 1 x y z xx xy xz yy yz zz xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz

// line along v_x at (j, k)
template <typename T, int N>
__device__ __forceinline__ void line_products(T (&m)[20], T S0, T S1, T S2, T S3, int j, int k) {
    const T c = T(0.5) * T(N - 1);
    T e = T(j) - c, z = T(k) - c;
    T e2 = e * e, z2 = z * z, ez = e * z;
    m[0] = S0; m[1] = S1; m[2] = e * S0; m[3] = z * S0;
    m[4] = S2; m[5] = e * S1; m[6] = z * S1; m[7] = e2 * S0; m[8] = ez * S0; m[9] = z2 * S0;
    m[10] = S3; m[11] = e * S2; m[12] = z * S2; m[13] = e2 * S1; m[14] = ez * S1; m[15] = z2 * S1;
    m[16] = e2 * e * S0; m[17] = e2 * z * S0; m[18] = e * z2 * S0; m[19] = z2 * z * S0;
}

// line along v_z at (i, j)
template <typename T, int N>
__device__ __forceinline__ void line_products_z(T (&m)[20], T S0, T S1, T S2, T S3, int i, int j) {
    const T c = T(0.5) * T(N - 1);
    const T x = T(i) - c, y = T(j) - c;
    const T x2 = x * x, y2 = y * y, xy = x * y;
    m[0] = S0; m[1] = x * S0; m[2] = y * S0; m[3] = S1;
    m[4] = x2 * S0; m[5] = xy * S0; m[6] = x * S1; m[7] = y2 * S0; m[8] = y * S1; m[9] = S2;
    m[10] = x2 * x * S0; m[11] = x2 * y * S0; m[12] = x2 * S1; m[13] = x * y2 * S0; m[14] = xy * S1;
    m[15] = x * S2; m[16] = y2 * y * S0; m[17] = y2 * S1; m[18] = y * S2; m[19] = S3;
}

// reduce the per-thread products over the CTA and write the 20 physical
// raw moments to out (uses red[20 * 32 + 20]; contains a __syncthreads).
// Warp partial sums are combined in T by lanes 0..19 of warp 0; only the
// final binomial expansion runs in FP64 (on GB300 an FP64 warp instruction
// occupies the pipe for many cycles however few lanes are active, so FP64
// work stays on one warp).
template <typename T>
__device__ __forceinline__ void reduce_moments(T (&m)[20], double* red, double* out, const MomConv& conv) {
    const int t = threadIdx.x;
#pragma unroll
    for (int a = 0; a < 20; ++a) {
        T v = m[a];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        m[a] = v;
    }
    const int warp = t >> 5, lane = t & 31, nwarp = blockDim.x >> 5;
    T* part = reinterpret_cast<T*>(red);
    if (lane == 0)
#pragma unroll
        for (int a = 0; a < 20; ++a) part[warp * 20 + a] = m[a];
    __syncthreads();
    double* im = red + 20 * 32;
    if (t < 20) {
        T sacc = T(0);
        for (int w = 0; w < nwarp; ++w) sacc += part[w * 20 + t];
        im[t] = (double)sacc;
    }
    __syncwarp();
    if (t < 20) {
        double acc = 0.0;
        for (int q = 0; q < conv.nterm[t]; ++q) acc += conv.coef[t][q] * im[conv.idx[t][q]];
        out[t] = acc;
    }
}

}  // namespace vl
