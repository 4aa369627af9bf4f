// Warm start of the moment fit by a small MLP (paper Sec. 2.2: the fitted
// discrete Maxwellians of Algorithm 1; the network only proposes the Newton
// start, Newton still converges to the same tolerance and falls back to the
// cold start).
//
// Per fit, 12 inputs from the fit targets (n, nu, E2 = int v v f) and the
// velocity box:
//   Theta_ab / (dv_a dv_b)            (xx, xy, xz, yy, yz, zz)
//   (u_a - v_nearest,a) / dv_a         offset of u from the nearest cell centre
//   (u_a - vmin_a) / (vmax_a - vmin_a) position of u in the box
// 10 outputs: eta* - eta_0, the Newton solution minus the cold start in the
// fit's scaled coordinates (w = (v - u0) / sigma), both dimensionless, so a
// network trained on one velocity grid applies to another.
// Network: 12 -> 128 -> 128 -> 10, GELU (erf form) on the hidden layers.
// Inputs are standardised (xm, xs). The outputs span many decades (most
// cells ~1e-5, Maxwellians cut by the velocity box ~1e-2), so the network
// predicts y_k = asinh(t_k / s_k), s_k the geometric mean of |t_k| over the
// training samples but at least 1e-6, the level of residual the cold start
// leaves anyway (linear for typical cells, logarithmic for large ones),
// centred by ym and scaled by ys = max(1, deviation) so that outputs that
// stay below that level (noise of the converged fits) weigh nothing;
// t_k = s_k sinh(y_k ys_k + ym_k).
//
// Parameter blob (FP32, VL_MLP_NPARAM floats; the layout of mlp_get_weights):
//   xm[12] xs[12] ym[10] ys[10] ysc[10] | W1[128][12] b1[128] | W2[128][128]
//   b2[128] | W3[10][128] b3[10]        (W[out][in], y = W x + b)
// Training samples (VL_MLP_SAMPLE floats each): x[12], t[10] (eta* - eta_0),
// flag (1 = usable), pad.
#pragma once

#include <cuda_runtime.h>

namespace vl {
namespace mlp {

constexpr int kIn = 12, kOut = 10, kHid = 128, kSample = 24;
constexpr int kOffXm = 0, kOffXs = 12, kOffYm = 24, kOffYs = 34, kOffYsc = 44;
constexpr int kNorm = 54;  // normalisation constants at the start of the blob
constexpr int kOffW1 = kNorm;
constexpr int kOffB1 = kOffW1 + kHid * kIn;
constexpr int kOffW2 = kOffB1 + kHid;
constexpr int kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid;
constexpr int kOffB3 = kOffW3 + kOut * kHid;
constexpr int kNParam = kOffB3 + kOut;
constexpr int kFirstTrained = kOffW1;  // normalisation constants are not trained
constexpr double kMinScale = 1e-6;    // smallest output scale s_k
// Out-of-distribution guard of the warm start (fits from targets only): a fit
// whose standardised inputs lie beyond kMaxInputSd, or whose standardised
// prediction lies beyond kMaxOutputSd, starts cold (the network has not seen
// such cells; a prediction far off sends Newton through slow evaluations).
constexpr float kMaxInputSd = 4.f, kMaxOutputSd = 6.f;

// Inputs of one fit from its targets t = (n, nu_x, nu_y, nu_z, E2_xx, E2_xy,
// E2_xz, E2_yy, E2_yz, E2_zz); false for targets the fit rejects.
__host__ __device__ inline bool fit_inputs(const double* t, const double* vmin, const double* dv, const double* vmax,
                                           float* x) {
    const double n = t[0];
    if (!(n > 0.0) || !(n < 1e300)) return false;
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = t[1 + a] / n;
    const int ab[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    for (int q = 0; q < 6; ++q) {
        const int a = ab[q][0], b = ab[q][1];
        const double th = t[4 + q] / n - u[a] * u[b];
        x[q] = (float)(th / (dv[a] * dv[b]));
    }
    if (!(x[0] > 0.f && x[3] > 0.f && x[5] > 0.f)) return false;
    for (int a = 0; a < 3; ++a) {
        const double ci = (u[a] - vmin[a]) / dv[a] - 0.5;
        const double near = vmin[a] + (floor(ci + 0.5) + 0.5) * dv[a];
        x[6 + a] = (float)((u[a] - near) / dv[a]);
        x[9 + a] = (float)((u[a] - vmin[a]) / (vmax[a] - vmin[a]));
    }
    for (int q = 0; q < kIn; ++q)
        if (!(x[q] == x[q]) || !(x[q] < 3.0e38f && x[q] > -3.0e38f)) return false;
    return true;
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

}  // namespace mlp
}  // namespace vl
