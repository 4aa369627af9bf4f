// Index helpers shared by the Newton fit kernels (newton.cuh: double-float
// on the FP32 pipe; newton64.cuh: FP64): packed monomials of degree <= 4 in
// three variables, packed lower triangles, the exponents of the ten basis
// functions phi = (1, w_x, w_y, w_z, w_x^2, w_x w_y, w_x w_z, w_y^2, w_y w_z,
// w_z^2) of the ten-moment Maxwellian (Sec. 2.2) and small binomials.
#pragma once

namespace vl {

// packed index of the monomial x^p y^q z^r, p + q + r <= 4 (by degree, then
// descending p, then descending q)
__host__ __device__ constexpr int mono4(int p, int q, int r) {
    int d = p + q + r, idx = 0;
    for (int e = 0; e < d; ++e) idx += (e + 1) * (e + 2) / 2;
    for (int pp = d; pp > p; --pp) idx += d - pp + 1;
    return idx + (d - p) - q;
}
// packed index of (i, j), j <= i, in a lower triangle
__host__ __device__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }
// exponent of w_axis in basis function a
__host__ __device__ constexpr int expo(int a, int axis) {
    return a == 0 ? 0
         : a <= 3 ? (a - 1 == axis ? 1 : 0)
         : a == 4 ? (axis == 0 ? 2 : 0)
         : a == 5 ? (axis <= 1 ? 1 : 0)
         : a == 6 ? (axis != 1 ? 1 : 0)
         : a == 7 ? (axis == 1 ? 2 : 0)
         : a == 8 ? (axis >= 1 ? 1 : 0)
         : (axis == 2 ? 2 : 0);
}
// packed index of (p, q), p + q <= 4 (by q, then p)
__host__ __device__ constexpr int tri4(int p, int q) {
    int idx = 0;
    for (int e = 0; e < q; ++e) idx += 5 - e;
    return idx + p;
}
// C(n, k) for n <= 4
__host__ __device__ constexpr int binom4(int n, int k) {
    return (k < 0 || k > n) ? 0 : (k == 0 || k == n) ? 1 : (k == 1 || k == n - 1) ? n : 6;
}

}  // namespace vl
