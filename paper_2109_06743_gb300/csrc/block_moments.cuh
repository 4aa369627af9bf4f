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
// raw moments to out (uses red[20 * MAXW + 20] for at most MAXW warps;
// contains a __syncthreads).
// Warp partial sums are combined in T by lanes 0..19 of warp 0; only the
// final binomial expansion runs in FP64 (on GB300 an FP64 warp instruction
// occupies the pipe for many cycles however few lanes are active, so FP64
// work stays on one warp).
//
// The warp stage is a reduce-scatter: at each of the five butterfly steps a
// lane keeps one half of its values (the lower or upper one, by the bit of
// its lane index) and adds the other half of its partner's, so 20 values
// take 10 + 5 + 3 + 2 + 1 shuffles instead of 5 each, and at the end lane
// L holds the warp sum of one moment (20 of the 32 lanes; the rest hold
// padding).
template <typename T>
__device__ __forceinline__ T rs_step(T keep_lo, T keep_hi, bool hi, int o) {
    const T send = hi ? keep_lo : keep_hi;
    return (hi ? keep_hi : keep_lo) + __shfl_xor_sync(0xffffffffu, send, o);
}

template <typename T, int MAXW = 32>
__device__ __forceinline__ void reduce_moments(T (&m)[20], double* red, double* out, const MomConv& conv) {
    const int t = threadIdx.x;
    const int warp = t >> 5, lane = t & 31, nwarp = blockDim.x >> 5;
    T a[10], b[5], c[3], d[2];
#pragma unroll
    for (int q = 0; q < 10; ++q) a[q] = rs_step<T>(m[q], m[10 + q], lane & 16, 16);  // moments hi*10 + q
#pragma unroll
    for (int q = 0; q < 5; ++q) b[q] = rs_step<T>(a[q], a[5 + q], lane & 8, 8);      // + (lane & 8 ? 5 : 0)
#pragma unroll
    for (int q = 0; q < 3; ++q) c[q] = rs_step<T>(b[q], q + 3 < 5 ? b[q + 3] : T(0), lane & 4, 4);
#pragma unroll
    for (int q = 0; q < 2; ++q) d[q] = rs_step<T>(c[q], q + 2 < 3 ? c[q + 2] : T(0), lane & 2, 2);
    const T e = rs_step<T>(d[0], d[1], lane & 1, 1);
    // the moment this lane now holds: groups of 10, 5, then 3 + 2 slots
    const int o = ((lane & 4) ? 3 : 0) + ((lane & 2) ? 2 : 0) + ((lane & 1) ? 1 : 0);
    const bool valid = o < ((lane & 4) ? 5 : 3);
    const int idx = ((lane & 16) ? 10 : 0) + ((lane & 8) ? 5 : 0) + o;
    T* part = reinterpret_cast<T*>(red);
    if (valid) part[warp * 20 + idx] = e;
    __syncthreads();
    double* im = red + 20 * MAXW;
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
