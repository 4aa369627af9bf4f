// Discrete ten-moment Maxwellian fit by Newton iteration in plain FP64
// (moment fitting, paper Sec. 2.2 and Algorithm 1): the FP64-mode fit. The
// FP32 mode uses the double-float kernel of newton.cuh instead.
//
// The fit is the one of the double-float kernel and of the oracle: unknowns
// are the natural parameters eta of M(v) = exp(eta . phi(w)) in scaled
// coordinates w_a = (v_a - u0_a) / sigma_a (u0 and sigma the targets' mean
// and standard deviations), the equations D(eta) = sum_c M(v_c) phi(w_c) dv^3
// = T are the gradient of a convex function whose Hessian is the Gram matrix
// sum M phi phi^T dv^3, the start and the fallback are the continuous
// Maxwellian of the targets, and each step is a full Newton step, damped by
// backtracking on the convex dual L(eta) = D_0 - eta . T while the residual
// exceeds 1e-6 n (Armijo factor 1e-4, at most 40 halvings).
//
// GB300 layout: one warp per cell (every branch of a fit is uniform over its
// warp). Lane L owns a contiguous run of the N^2 v_x lines of the block.
// Along a v_x line the exponent is quadratic in the cell index, so M follows
// the multiplicative recurrence M <- M r, r <- r exp(2 k_xx); line starts
// follow the same recurrence along v_y and restart (three exponentials) at
// the lane's first line and at every new v_z plane. The weights are the
// centred indices c = i - (N-1)/2, which the unrolled line loop holds as
// constants, so a cell costs five FP64 operations (seven with the Gram
// sums). Sums are reduced by xor butterflies (identical bits in every lane).
// The Gram sums of degree <= 4 give the Jacobian through three separable
// binomial transforms; lane 0 solves the 10 x 10 system by Cholesky.
// Blocks whose exponent leaves +-700 at a corner of the box, or whose
// one-cell ratios leave that range, take one exponential per cell instead.
#pragma once

#include "common.cuh"
#include "fit_index.cuh"
#include "kernels.cuh"
#include "mlp_common.cuh"

namespace vl {
namespace fit64 {
namespace {

constexpr int kCoefN = 16;
constexpr int kCellsPerCta = 4;  // one warp per cell

struct Cell {
    double eta[10], et[10], eta0[10], T[10], step[10];
    double m[10];   // index moments of degree <= 2 about the box centre
    double g[35];   // index moments of degree <= 4 (Gram sums)
    double k[10];   // index-space exponent of the last evaluation
    double wc[3], h[3], u0[3], sg[3];
    double tgt[10];
    // Newton step scratch: binomial coefficients of the three axes, the
    // transformed Gram sums, the packed Jacobian and its factor's pivots
    double cb[3][15], U[35], W[35], J[55], dinv[10];
};

// inverse of mono4: the exponents (p, q, r) of packed monomial m
__device__ __forceinline__ void mono4_exps(int m, int& p, int& q, int& r) {
    p = q = r = 0;
#pragma unroll 1
    for (int a = 0; a <= 4; ++a)
#pragma unroll 1
        for (int b = 0; b <= 4 - a; ++b)
#pragma unroll 1
            for (int c = 0; c <= 4 - a - b; ++c)
                if (mono4(a, b, c) == m) {
                    p = a;
                    q = b;
                    r = c;
                }
}
// inverse of tri: (i, j), j <= i, of packed index e
__device__ __forceinline__ void tri_ij(int e, int& i, int& j) {
    i = 0;
    while (tri(i + 1, 0) <= e) ++i;
    j = e - tri(i, 0);
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ double warp_allsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// index-space exponent q(c) = k0 + k_a c_a + k_ab c_a c_b of eta, with
// w_a = wc_a + h_a c_a (c the centred cell indices)
__device__ __forceinline__ void index_coeffs64(const double* e, const double* wc, const double* h, double* k) {
    k[0] = e[0] + e[1] * wc[0] + e[2] * wc[1] + e[3] * wc[2] + e[4] * wc[0] * wc[0] + e[5] * wc[0] * wc[1] +
           e[6] * wc[0] * wc[2] + e[7] * wc[1] * wc[1] + e[8] * wc[1] * wc[2] + e[9] * wc[2] * wc[2];
    k[1] = h[0] * (e[1] + 2.0 * e[4] * wc[0] + e[5] * wc[1] + e[6] * wc[2]);
    k[2] = h[1] * (e[2] + 2.0 * e[7] * wc[1] + e[5] * wc[0] + e[8] * wc[2]);
    k[3] = h[2] * (e[3] + 2.0 * e[9] * wc[2] + e[6] * wc[0] + e[8] * wc[1]);
    k[4] = e[4] * h[0] * h[0];
    k[5] = e[5] * h[0] * h[1];
    k[6] = e[6] * h[0] * h[2];
    k[7] = e[7] * h[1] * h[1];
    k[8] = e[8] * h[1] * h[2];
    k[9] = e[9] * h[2] * h[2];
}

// Can the recurrences represent every value and one-cell ratio of the block
// in normal FP64 numbers? The exponent at every corner above -700 (a
// quadratic with concave diagonal is smallest at a corner; if a diagonal
// coefficient is not negative the block is refused) and every one-cell
// difference along x and y, and the ratio multipliers, within +-700
// (differences are linear in position, extreme at the corners).
template <int N>
__device__ bool recurrence_ok(const double* k) {
    const int l = lane_id() & 7;
    constexpr double hN = 0.5 * (N - 1);
    bool ok = k[4] < 0.0 && k[7] < 0.0 && k[9] < 0.0 && fabs(2.0 * k[4]) < 700.0 && fabs(2.0 * k[7]) < 700.0 &&
              fabs(k[5]) < 700.0;
    const double x = (l & 1) ? hN : -hN, y = (l & 2) ? hN : -hN, z = (l & 4) ? hN : -hN;
    const double q = k[0] + k[1] * x + k[2] * y + k[3] * z + k[4] * x * x + k[5] * x * y + k[6] * x * z +
                     k[7] * y * y + k[8] * y * z + k[9] * z * z;
    ok = ok && q > -700.0 && q < 700.0;
    const double dx = k[4] * (2.0 * x + 1.0) + k[1] + k[5] * y + k[6] * z;
    const double dy = k[7] * (2.0 * y + 1.0) + k[2] + k[5] * x + k[8] * z;
    ok = ok && fabs(dx) < 700.0 && fabs(dy) < 700.0;
    return __all_sync(0xffffffffu, ok);
}

// The block's sums are accumulated per plane: over a lane's run of lines in
// one v_z plane the z index ck is constant, so a line's sums S_p = sum_i
// c_i^p M are first summed with the powers of the y index cj (P: S0, S1, S2,
// cj S0, cj S1, cj^2 S0; G[p][q] = sum S_p cj^q, p + q <= 4), and at the end
// of the run those times the powers of ck go into the ten moments m and the
// 35 Gram sums g.
template <bool GRAM>
__device__ __forceinline__ void plane_add64(double (&P)[6], double (&G)[GRAM ? 15 : 1], const double (&S)[5],
                                            double cj) {
    P[0] += S[0];
    P[1] += S[1];
    P[2] += S[2];
    P[3] = fma(cj, S[0], P[3]);
    P[4] = fma(cj, S[1], P[4]);
    P[5] = fma(cj * cj, S[0], P[5]);
    if (GRAM) {
        double pj = 1.0;
#pragma unroll
        for (int q = 0; q <= 4; ++q) {
#pragma unroll
            for (int pp = 0; pp <= 4 - q; ++pp) G[tri4(pp, q)] = fma(S[pp], pj, G[tri4(pp, q)]);
            pj *= cj;
        }
    }
}

template <bool GRAM>
__device__ __forceinline__ void plane_flush64(double (&m)[10], double (&g)[GRAM ? 35 : 1], double (&P)[6],
                                              double (&G)[GRAM ? 15 : 1], double ck) {
    m[0] += P[0];
    m[1] += P[1];
    m[2] += P[3];
    m[3] = fma(ck, P[0], m[3]);
    m[4] += P[2];
    m[5] += P[4];
    m[6] = fma(ck, P[1], m[6]);
    m[7] += P[5];
    m[8] = fma(ck, P[3], m[8]);
    m[9] = fma(ck * ck, P[0], m[9]);
#pragma unroll
    for (int q = 0; q < 6; ++q) P[q] = 0.0;
    if (GRAM) {
        double pk = 1.0;
#pragma unroll
        for (int r = 0; r <= 4; ++r) {
#pragma unroll
            for (int pp = 0; pp <= 4 - r; ++pp)
#pragma unroll
                for (int q = 0; q <= 4 - r - pp; ++q) g[mono4(pp, q, r)] = fma(G[tri4(pp, q)], pk, g[mono4(pp, q, r)]);
            pk *= ck;
        }
#pragma unroll
        for (int q = 0; q < 15; ++q) G[q] = 0.0;
    }
}

// Reduce-scatter of NV values (a multiple of 16) over the warp: after the
// four steps of exchange distance 16, 8, 4, 2 a lane holds NV/16 partial sums
// (the half picked by each lane bit in turn); the last step (distance 1)
// adds the partner's values whole, so v[0 .. NV/16 - 1] of lanes L and L^1
// are the warp sums of values (bit4 NV/2 + bit3 NV/4 + bit2 NV/8 + bit1 NV/16)
// + 0 .. NV/16 - 1.
template <int NV>
__device__ __forceinline__ void reduce_scatter64(double (&v)[NV], int lane) {
#pragma unroll
    for (int lvl = 0; lvl < 4; ++lvl) {
        const int o = 16 >> lvl, h = NV >> (lvl + 1);
        const bool hi = (lane & o) != 0;
#pragma unroll
        for (int q = 0; q < h; ++q) {
            const double keep = hi ? v[h + q] : v[q];
            const double send = hi ? v[q] : v[h + q];
            v[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
#pragma unroll
    for (int q = 0; q < NV / 16; ++q) v[q] += __shfl_xor_sync(0xffffffffu, v[q], 1);
}

// Index moments (cs.m; with GRAM also the Gram sums cs.g) of M = exp(q(c))
// over the block. Returns false if any sum is not finite.
template <int N, bool GRAM>
__device__ __noinline__ bool eval64(Cell& cs) {
    const int lane = lane_id();
    constexpr double hN = 0.5 * (N - 1);
    constexpr int NL = N * N;
    const int l0 = (lane * NL) >> 5, l1 = ((lane + 1) * NL) >> 5;
    double k[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) k[q] = cs.k[q];
    double m[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) m[q] = 0.0;
    double g[GRAM ? 35 : 1], P[6], G[GRAM ? 15 : 1];
#pragma unroll
    for (int q = 0; q < (GRAM ? 35 : 1); ++q) g[q] = 0.0;
#pragma unroll
    for (int q = 0; q < 6; ++q) P[q] = 0.0;
#pragma unroll
    for (int q = 0; q < (GRAM ? 15 : 1); ++q) G[q] = 0.0;
    if (recurrence_ok<N>(k)) {
        const double e_in = exp(2.0 * k[4]), e_j = exp(2.0 * k[7]), e_xy = exp(k[5]);
        double Ms = 0.0, rs = 0.0, rl = 0.0;
#pragma unroll 1
        for (int l = l0; l < l1; ++l) {
            const int j = l % N, kk = l / N;
            const double cj = j - hN, ck = kk - hN;
            if (l == l0 || j == 0) {
                // q along the line: k_xx c^2 + B c + C
                const double B = k[1] + k[5] * cj + k[6] * ck;
                const double C = k[0] + k[2] * cj + k[3] * ck + k[7] * cj * cj + k[8] * cj * ck + k[9] * ck * ck;
                Ms = exp((k[4] * hN - B) * hN + C);
                rs = exp(k[4] * (2.0 - N) + B);
                rl = exp(k[2] - k[5] * hN + k[7] * (2.0 * cj + 1.0) + k[8] * ck);
            }
            double S[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
            double M = Ms, r = rs;
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const double c = i - hN;
                S[0] += M;
                S[1] = fma(M, c, S[1]);
                S[2] = fma(M, c * c, S[2]);
                if (GRAM) {
                    S[3] = fma(M, c * c * c, S[3]);
                    S[4] = fma(M, c * c * c * c, S[4]);
                }
                M *= r;
                r *= e_in;
            }
            plane_add64<GRAM>(P, G, S, cj);
            if (j == N - 1 || l == l1 - 1) plane_flush64<GRAM>(m, g, P, G, ck);
            Ms *= rl;
            rl *= e_j;
            rs *= e_xy;
        }
    } else {
        // one exponential per cell (any exponent range)
#pragma unroll 1
        for (int l = l0; l < l1; ++l) {
            const int j = l % N, kk = l / N;
            const double cj = j - hN, ck = kk - hN;
            const double B = k[1] + k[5] * cj + k[6] * ck;
            const double C = k[0] + k[2] * cj + k[3] * ck + k[7] * cj * cj + k[8] * cj * ck + k[9] * ck * ck;
            double S[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll 4
            for (int i = 0; i < N; ++i) {
                const double c = i - hN;
                const double M = exp((k[4] * c + B) * c + C);
                S[0] += M;
                S[1] = fma(M, c, S[1]);
                S[2] = fma(M, c * c, S[2]);
                if (GRAM) {
                    S[3] = fma(M, c * c * c, S[3]);
                    S[4] = fma(M, c * c * c * c, S[4]);
                }
            }
            plane_add64<GRAM>(P, G, S, cj);
            if (j == N - 1 || l == l1 - 1) plane_flush64<GRAM>(m, g, P, G, ck);
        }
    }
    // warp sums by reduce-scatter: the 10 moments (and 35 Gram sums), padded
    // to 16 (48), are halved at each of four exchange steps (a lane keeps the
    // half its lane bit selects and adds its partner's copy of that half),
    // then the last step adds the partner's whole remainder; lanes L and L^1
    // end with the same 1 (3) sums, which the even lane stores. 16 (48)
    // additions per lane instead of 50 (225) for a butterfly per value.
    bool fin = true;
    if (GRAM) {
        double v[48];
#pragma unroll
        for (int q = 0; q < 48; ++q) v[q] = q < 10 ? m[q] : (q < 45 ? g[q - 10] : 0.0);
        reduce_scatter64<48>(v, lane);
        const int base = ((lane >> 4) & 1) * 24 + ((lane >> 3) & 1) * 12 + ((lane >> 2) & 1) * 6 + ((lane >> 1) & 1) * 3;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int idx = base + q;
            fin = fin && (idx >= 45 || isfinite(v[q]));
            if ((lane & 1) == 0 && idx < 45) {
                if (idx < 10) cs.m[idx] = v[q];
                else cs.g[idx - 10] = v[q];
            }
        }
    } else {
        double v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = q < 10 ? m[q] : 0.0;
        reduce_scatter64<16>(v, lane);
        const int idx = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
        fin = idx >= 10 || isfinite(v[0]);
        if ((lane & 1) == 0 && idx < 10) cs.m[idx] = v[0];
    }
    fin = __all_sync(0xffffffffu, fin);
    __syncwarp();
    return fin;
}

// evaluation at eta (cs.k set from it); returns whether the sums are finite
template <int N>
__device__ __forceinline__ bool evaluate64(Cell& cs, const double* eta, bool gram) {
    if (lane_id() == 0) index_coeffs64(eta, cs.wc, cs.h, cs.k);
    __syncwarp();
    return gram ? eval64<N, true>(cs) : eval64<N, false>(cs);
}

// w-space moments D (10) from the index moments about the box centre
__device__ __forceinline__ void w_moments64(const Cell& cs, double vol, double* D) {
    const double* m = cs.m;
    const double* w = cs.wc;
    const double* h = cs.h;
    D[0] = m[0];
    D[1] = w[0] * m[0] + h[0] * m[1];
    D[2] = w[1] * m[0] + h[1] * m[2];
    D[3] = w[2] * m[0] + h[2] * m[3];
    D[4] = w[0] * w[0] * m[0] + 2.0 * w[0] * h[0] * m[1] + h[0] * h[0] * m[4];
    D[5] = w[0] * w[1] * m[0] + w[0] * h[1] * m[2] + h[0] * w[1] * m[1] + h[0] * h[1] * m[5];
    D[6] = w[0] * w[2] * m[0] + w[0] * h[2] * m[3] + h[0] * w[2] * m[1] + h[0] * h[2] * m[6];
    D[7] = w[1] * w[1] * m[0] + 2.0 * w[1] * h[1] * m[2] + h[1] * h[1] * m[7];
    D[8] = w[1] * w[2] * m[0] + w[1] * h[2] * m[3] + h[1] * w[2] * m[2] + h[1] * h[2] * m[8];
    D[9] = w[2] * w[2] * m[0] + 2.0 * w[2] * h[2] * m[3] + h[2] * h[2] * m[9];
#pragma unroll
    for (int q = 0; q < 10; ++q) D[q] *= vol;
}

// Newton direction, with the warp's lanes sharing the work (an FP64 warp
// instruction costs the FP64 pipe the same with one lane active as with
// 32): the binomial coefficients of (w + h c)^A per axis, the Gram matrix
// in w-space from the index sums by three separable transforms (one
// output per lane), an LDL^T factorisation whose column updates run one
// entry per lane, and the two triangular solves with one unknown per lane.
// Returns (to every lane) whether J was positive definite.
__device__ __noinline__ bool newton_step64(Cell& cs, const double* G, double vol) {
    const int lane = lane_id();
    if (lane < 15) {
        int A, pp;
        tri_ij(lane, A, pp);
        const double bn = (double)binom4(A, pp);
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            double v = bn;
            for (int e = 0; e < A - pp; ++e) v *= cs.wc[ax];
            for (int e = 0; e < pp; ++e) v *= cs.h[ax];
            cs.cb[ax][lane] = v;
        }
    }
    __syncwarp();
    // x: U[A, q, r] = sum_p c_x[A][p] g[p, q, r]
    for (int m = lane; m < 35; m += 32) {
        int A, q, r;
        mono4_exps(m, A, q, r);
        double acc = 0.0;
        for (int pp = 0; pp <= A; ++pp) acc = fma(cs.cb[0][tri(A, pp)], cs.g[mono4(pp, q, r)], acc);
        cs.U[m] = acc;
    }
    __syncwarp();
    // y: W[A, B, r] = sum_q c_y[B][q] U[A, q, r]
    for (int m = lane; m < 35; m += 32) {
        int A, B, r;
        mono4_exps(m, A, B, r);
        double acc = 0.0;
        for (int q = 0; q <= B; ++q) acc = fma(cs.cb[1][tri(B, q)], cs.U[mono4(A, q, r)], acc);
        cs.W[m] = acc;
    }
    __syncwarp();
    // z: U[A, B, C] = vol sum_r c_z[C][r] W[A, B, r]
    for (int m = lane; m < 35; m += 32) {
        int A, B, C;
        mono4_exps(m, A, B, C);
        double acc = 0.0;
        for (int r = 0; r <= C; ++r) acc = fma(cs.cb[2][tri(C, r)], cs.W[mono4(A, B, r)], acc);
        cs.U[m] = acc * vol;
    }
    __syncwarp();
    for (int e = lane; e < 55; e += 32) {
        int ia, ib;
        tri_ij(e, ia, ib);
        cs.J[e] = cs.U[mono4(expo(ia, 0) + expo(ib, 0), expo(ia, 1) + expo(ib, 1), expo(ia, 2) + expo(ib, 2))];
    }
    __syncwarp();
    // LDL^T, right-looking: column j's pivot d_j, multipliers l_ij = a_ij / d_j
    // (stored in place), then the trailing update a_ik -= l_ij d_j l_kj
    bool ok = true;
    for (int j = 0; j < 10; ++j) {
        const double d = cs.J[tri(j, j)];
        ok = ok && d > 0.0;
        const double di = 1.0 / fmax(d, 1e-300);
        double lij = 0.0;
        if (lane > j && lane < 10) lij = cs.J[tri(lane, j)] * di;
        __syncwarp();
        for (int e = lane; e < 55; e += 32) {
            int i, k;
            tri_ij(e, i, k);
            if (k > j) cs.J[e] -= cs.J[tri(i, j)] * cs.J[tri(k, j)] * di;
        }
        __syncwarp();
        if (lane > j && lane < 10) cs.J[tri(lane, j)] = lij;
        if (lane == 0) cs.dinv[j] = di;
        __syncwarp();
    }
    // L y = -G (unit diagonal), D z = y, L^T x = z; unknown i on lane i
    double b = lane < 10 ? -G[lane] : 0.0;
    for (int i = 0; i < 10; ++i) {
        const double yi = __shfl_sync(0xffffffffu, b, i);
        if (lane > i && lane < 10) b = fma(-cs.J[tri(lane, i)], yi, b);
    }
    if (lane < 10) b *= cs.dinv[lane];
    for (int i = 9; i >= 0; --i) {
        const double xi = __shfl_sync(0xffffffffu, b, i);
        if (lane < i) b = fma(-cs.J[tri(i, lane)], xi, b);
    }
    if (lane < 10) cs.step[lane] = b;
    __syncwarp();
    return __all_sync(0xffffffffu, ok);
}

// Fit set-up (lane 0, targets in cs.tgt): scaled coordinates, w-space
// targets T = (n, 0, n Corr) and the continuous Maxwellian eta0. Returns
// (to every lane) false for invalid targets (n <= 0 or not finite, Theta not
// positive definite).
template <int N>
__device__ __noinline__ bool setup64(Cell& cs, const FitArgs& a) {
    int ok = 0;
    if (lane_id() == 0) {
        const double* t = cs.tgt;
        const double n = t[0];
        if (n > 0.0 && isfinite(n)) {
            double u0[3], Th[9];
            for (int q = 0; q < 3; ++q) u0[q] = t[1 + q] / n;
            const int pk[3][3] = {{4, 5, 6}, {5, 7, 8}, {6, 8, 9}};
            for (int p = 0; p < 3; ++p)
                for (int q = 0; q < 3; ++q) Th[p * 3 + q] = t[pk[p][q]] / n - u0[p] * u0[q];
            // positive definite (Cholesky)
            bool pd = Th[0] > 0.0;
            double l00 = 0, l10 = 0, l20 = 0, l11 = 0, l21 = 0;
            if (pd) {
                l00 = sqrt(Th[0]);
                l10 = Th[3] / l00;
                l20 = Th[6] / l00;
                const double d1 = Th[4] - l10 * l10;
                pd = d1 > 0.0;
                if (pd) {
                    l11 = sqrt(d1);
                    l21 = (Th[7] - l20 * l10) / l11;
                    pd = Th[8] - l20 * l20 - l21 * l21 > 0.0;
                }
            }
            bool fin = true;
            for (int q = 0; q < 10; ++q) fin = fin && isfinite(t[q]);
            if (pd && fin) {
                double sg[3], Cr[9];
                for (int q = 0; q < 3; ++q) sg[q] = sqrt(Th[q * 4]);
                for (int p = 0; p < 3; ++p)
                    for (int q = 0; q < 3; ++q) Cr[p * 3 + q] = Th[p * 3 + q] / (sg[p] * sg[q]);
                for (int q = 0; q < 3; ++q) {
                    cs.u0[q] = u0[q];
                    cs.sg[q] = sg[q];
                    cs.h[q] = a.dv[q] / sg[q];
                    cs.wc[q] = (a.vmin[q] + 0.5 * N * a.dv[q] - u0[q]) / sg[q];
                }
                cs.T[0] = n;
                cs.T[1] = cs.T[2] = cs.T[3] = 0.0;
                cs.T[4] = n * Cr[0];
                cs.T[5] = n * Cr[1];
                cs.T[6] = n * Cr[2];
                cs.T[7] = n * Cr[4];
                cs.T[8] = n * Cr[5];
                cs.T[9] = n * Cr[8];
                // P = Corr^-1
                const double c00 = Cr[4] * Cr[8] - Cr[5] * Cr[7], c01 = Cr[5] * Cr[6] - Cr[3] * Cr[8],
                             c02 = Cr[3] * Cr[7] - Cr[4] * Cr[6];
                const double id = 1.0 / (Cr[0] * c00 + Cr[1] * c01 + Cr[2] * c02);
                const double P00 = c00 * id, P01 = (Cr[2] * Cr[7] - Cr[1] * Cr[8]) * id,
                             P02 = (Cr[1] * Cr[5] - Cr[2] * Cr[4]) * id, P11 = (Cr[0] * Cr[8] - Cr[2] * Cr[6]) * id,
                             P12 = (Cr[2] * Cr[3] - Cr[0] * Cr[5]) * id, P22 = (Cr[0] * Cr[4] - Cr[1] * Cr[3]) * id;
                const double detTh = Th[0] * (Th[4] * Th[8] - Th[5] * Th[7]) - Th[1] * (Th[3] * Th[8] - Th[5] * Th[6]) +
                                     Th[2] * (Th[3] * Th[7] - Th[4] * Th[6]);
                cs.eta0[0] = log(n) - 1.5 * log(2.0 * 3.14159265358979323846) - 0.5 * log(detTh);
                cs.eta0[1] = cs.eta0[2] = cs.eta0[3] = 0.0;
                cs.eta0[4] = -0.5 * P00;
                cs.eta0[5] = -P01;
                cs.eta0[6] = -P02;
                cs.eta0[7] = -0.5 * P11;
                cs.eta0[8] = -P12;
                cs.eta0[9] = -0.5 * P22;
                ok = 1;
            }
        }
    }
    __syncwarp();
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// the fitted exponent must be a Gaussian: -2 mu positive definite
__device__ __forceinline__ bool gaussian64(const double* e) {
    const double a00 = -2.0 * e[4], a10 = -e[5], a20 = -e[6], a11 = -2.0 * e[7], a21 = -e[8], a22 = -2.0 * e[9];
    if (!(a00 > 0.0)) return false;
    const double l00 = sqrt(a00), l10 = a10 / l00, l20 = a20 / l00, d1 = a11 - l10 * l10;
    if (!(d1 > 0.0)) return false;
    const double l11 = sqrt(d1), l21 = (a21 - l20 * l10) / l11;
    return a22 - l20 * l20 - l21 * l21 > 0.0;
}

struct Work64 {
    unsigned m, g, warm;
};

// Newton iteration from cs.eta (uniform over the warp). Returns whether the
// residual reached tol n and the fitted exponent is a Gaussian; *iters gets
// the number of Newton steps.
template <int N>
__device__ __noinline__ bool newton64(Cell& cs, const FitArgs& a, double n, double vol, int* iters, Work64& work) {
    const int lane = lane_id();
    const double tol = a.tol * n;
    bool haveD = false, haveG = false, gram_next = true, converged = false;
    int it = 0;
    for (it = 0;; ++it) {
        if (!haveD) {
            evaluate64<N>(cs, cs.eta, gram_next);
            work.m += 1u;
            work.g += gram_next ? 1u : 0u;
            haveD = true;
            haveG = gram_next;
        }
        double D[10], G[10];
        w_moments64(cs, vol, D);
        double gmax = 0.0;
        bool fin = true;
#pragma unroll
        for (int q = 0; q < 10; ++q) {
            G[q] = D[q] - cs.T[q];
            fin = fin && isfinite(G[q]);
            gmax = fmax(gmax, fabs(G[q]));
        }
        if (fin && gmax <= tol) {
            converged = true;
            break;
        }
        if (!fin || it == a.max_iter) break;
        if (!haveG) {
            // the Jacobian at eta (the moments come out the same)
            evaluate64<N>(cs, cs.eta, true);
            work.m += 1u;
            work.g += 1u;
            haveG = true;
        }
        if (!newton_step64(cs, G, vol)) break;
        const double rel = gmax / n;
        // Gram sums with the next evaluation where another step is likely
        // (the residual after a Newton step falls roughly as its square)
        gram_next = 100.0 * rel * rel > a.tol;
        if (gmax > 1e-6 * n) {
            double L0 = D[0], gd = 0.0;
#pragma unroll
            for (int q = 0; q < 10; ++q) {
                L0 -= cs.eta[q] * cs.T[q];
                gd += G[q] * cs.step[q];
            }
            double lam = 1.0;
            bool accepted = false;
            for (int ls = 0; ls < 40; ++ls) {
                if (lane < 10) cs.et[lane] = cs.eta[lane] + lam * cs.step[lane];
                __syncwarp();
                const bool ef = evaluate64<N>(cs, cs.et, gram_next);
                work.m += 1u;
                work.g += gram_next ? 1u : 0u;
                double L1 = cs.m[0] * vol;
#pragma unroll
                for (int q = 0; q < 10; ++q) L1 -= cs.et[q] * cs.T[q];
                if (ef && isfinite(L1) && L1 <= L0 + 1e-4 * lam * gd) {
                    accepted = true;
                    break;
                }
                lam *= 0.5;
            }
            if (lane < 10) cs.eta[lane] = accepted ? cs.et[lane] : cs.eta[lane] + lam * cs.step[lane];
            __syncwarp();
            haveD = accepted;
            haveG = accepted && gram_next;
        } else {
            if (lane < 10) cs.eta[lane] = cs.eta[lane] + cs.step[lane];
            __syncwarp();
            haveD = false;
            haveG = false;
        }
    }
    *iters = it;
    return converged && gaussian64(cs.eta);
}

// non-finite or negative targets (a numeric error upstream); empty cells
// (n = 0) are not
__device__ __forceinline__ bool bad_targets(const double* t, int n) {
    bool bad = !(t[0] >= 0.0);
    for (int q = 0; q < n; ++q) bad = bad || !isfinite(t[q]);
    return bad;
}

// One fit by a warp: from the network's prediction when warm is not null
// (then from the cold start if that run fails), else from the continuous
// Maxwellian. Writes the coefficients (eta, u0, sigma) to coef, appends a
// training sample of a converged fit when harvesting; returns 0 converged,
// 1 fallback (continuous Maxwellian), 2 invalid targets.
template <int N>
__device__ int fit_cell64(Cell& cs, const FitArgs& a, double* coef, const float* warm, int* iters, Work64& work) {
    const int lane = lane_id();
    *iters = 0;
    if (!setup64<N>(cs, a)) {
        if (lane < kCoefN) coef[lane] = 0.0;
        return 2;
    }
    const double n = cs.tgt[0];
    const double vol = a.dv[0] * a.dv[1] * a.dv[2];
    bool good = false;
    // the guard of the network's inference writes NaN rows for the fits it rejects
    if (warm && warm[0] == warm[0] && fabsf(warm[0]) < 1e30f) work.warm += 1u;
    if (warm) {
        if (lane < 10) {
            const float dw = warm[lane];
            cs.eta[lane] = cs.eta0[lane] + ((dw == dw && fabsf(dw) < 1e30f) ? (double)dw : 0.0);
        }
        __syncwarp();
        good = newton64<N>(cs, a, n, vol, iters, work);
    }
    if (!good) {
        if (lane < 10) cs.eta[lane] = cs.eta0[lane];
        __syncwarp();
        int it2 = 0;
        good = newton64<N>(cs, a, n, vol, &it2, work);
        *iters += it2;
    }
    if (lane < 10) coef[lane] = good ? cs.eta[lane] : cs.eta0[lane];
    else if (lane < 13) coef[lane] = cs.u0[lane - 10];
    else if (lane < 16) coef[lane] = cs.sg[lane - 13];
    if (good && a.harvest) {
        unsigned long long slot = 0;
        if (lane == 0) slot = atomicAdd(a.harvest_count, 1ull);
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (slot < (unsigned long long)a.harvest_cap) {
            float* smp = a.harvest + slot * mlp::kSample;
            if (lane == 0) {
                float x[mlp::kIn];
                const bool ok = mlp::fit_inputs(cs.tgt, a.vmin, a.dv, a.vmax, x);
                for (int q = 0; q < mlp::kIn; ++q) smp[q] = x[q];
                smp[22] = ok ? 1.f : 0.f;
                smp[23] = 0.f;
            }
            if (lane < 10) smp[mlp::kIn + lane] = (float)(cs.eta[lane] - cs.eta0[lane]);
        }
    }
    __syncwarp();
    return good ? 0 : 1;
}

template <int N>
__global__ void __launch_bounds__(32 * kCellsPerCta) newton64_kernel(FitArgs a) {
    __shared__ Cell cells[kCellsPerCta];
    __shared__ unsigned long long cnt[VL_NSTATS];
    if (threadIdx.x < VL_NSTATS) cnt[threadIdx.x] = 0ull;
    __syncthreads();
    const int lane = lane_id();
    const int slot = threadIdx.x >> 5;
    Cell& cs = cells[slot];
    for (long long cell = (long long)blockIdx.x * kCellsPerCta + slot; cell < a.ncell;
         cell += (long long)gridDim.x * kCellsPerCta) {
        // V targets: the moments of f
        if (lane < 10) cs.tgt[lane] = a.vmom[cell * 20 + lane];
        __syncwarp();
        bool bad = lane == 0 && bad_targets(cs.tgt, 10);
        const double nV = cs.tgt[0];
        Work64 work = {0u, 0u, 0u};
        int itv = 0, itf = 0;
        const float* wv = a.warm ? a.warm + cell * 20 : nullptr;
        const int stv = fit_cell64<N>(cs, a, a.coef_v + cell * kCoefN, wv, &itv, work);
        // F targets: the fluid moments rescaled by n_V / n_F
        const double nF = a.fluid[cell * 10];
        if (lane == 0) {
            double raw[10];
            for (int q = 0; q < 10; ++q) raw[q] = a.fluid[cell * 10 + q];
            bad = bad || bad_targets(raw, 10);
        }
        const double scale = nF > 0.0 ? nV / nF : 0.0;
        __syncwarp();
        if (lane < 10) {
            cs.tgt[lane] = a.fluid[cell * 10 + lane] * scale;
        }
        __syncwarp();
        if (lane < 10) a.fluid[cell * 10 + lane] = cs.tgt[lane];
        const float* wf = a.warm ? a.warm + cell * 20 + 10 : nullptr;
        const int stf = fit_cell64<N>(cs, a, a.coef_f + cell * kCoefN, wf, &itf, work);
        if (lane == 0) {
            a.status[cell * 2] = stv;
            a.status[cell * 2 + 1] = stf;
            if (bad && a.numeric) *reinterpret_cast<volatile int*>(a.numeric) = VL_ENUMERIC;
            atomicAdd_block(&cnt[CNT_ITERS], (unsigned long long)(itv + itf));
            const unsigned long long fb = (stv == 1) + (stf == 1);
            if (fb) atomicAdd_block(&cnt[CNT_FALLBACK], fb);
            const unsigned long long inv = (stv == 2) + (stf == 2);
            if (inv) atomicAdd_block(&cnt[CNT_INVALID], inv);
            atomicAdd_block(&cnt[CNT_EVAL64_M], (unsigned long long)work.m);
            atomicAdd_block(&cnt[CNT_EVAL64_G], (unsigned long long)work.g);
            if (work.warm) atomicAdd_block(&cnt[CNT_WARM], (unsigned long long)work.warm);
        }
        __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x < VL_NSTATS && threadIdx.x != CNT_CLIPPED && cnt[threadIdx.x])
        atomicAdd(&a.counters[threadIdx.x], cnt[threadIdx.x]);
}

template <int N>
cudaError_t launch64(const FitArgs& a, cudaStream_t st) {
    long long blocks = (a.ncell + kCellsPerCta - 1) / kCellsPerCta;
    if (blocks > 0x7FFFFFFFLL) blocks = 0x7FFFFFFFLL;
    if (blocks < 1) return cudaSuccess;
    newton64_kernel<N><<<(unsigned)blocks, 32 * kCellsPerCta, 0, st>>>(a);
    count_launch();
    return cudaGetLastError();
}

}  // namespace
}  // namespace fit64
}  // namespace vl
