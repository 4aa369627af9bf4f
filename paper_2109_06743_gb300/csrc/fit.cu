// Moment fitting (paper Sec. 2.2, Algorithm 1 "Moment Fitting"): the
// exchange of the fitted Maxwellians and the limiter, the 1D1V fits, and the
// conversion of fit coefficients to the paper's parameters. The 2D3V Newton
// fits are in newton.cu.
//
// exchange_kernel: f <- f - f_M,V + f_M,F, clip negative values and rescale
// the cell to n_V (limiter of Algorithm 1), fused with the moments of the
// new f; the Maxwellians' line parameters come from exchange_params_kernel.
#include "common.cuh"
#include "kernels.cuh"
#include "block_moments.cuh"

namespace vl {

constexpr int kCoef = 16;  // per fit: eta[10], u0[3], sigma[3]

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return __shfl_sync(0xffffffffu, v, 0);
}

__device__ __forceinline__ double bcast(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ float bcastf(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }

// 3x3 symmetric helpers (row-major)
__device__ bool chol3(const double* A, double* L) {
    for (int i = 0; i < 9; ++i) L[i] = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = A[i * 3 + j];
            for (int k = 0; k < j; ++k) s -= L[i * 3 + k] * L[j * 3 + k];
            if (i == j) {
                if (!(s > 0.0)) return false;
                L[i * 3 + i] = sqrt(s);
            } else {
                L[i * 3 + j] = s / L[j * 3 + j];
            }
        }
    return true;
}

__device__ void inv3(const double* A, double* I) {
    double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
    double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    double id = 1.0 / det;
    I[0] = c00 * id;
    I[1] = (A[2] * A[7] - A[1] * A[8]) * id;
    I[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    I[3] = c01 * id;
    I[4] = (A[0] * A[8] - A[2] * A[6]) * id;
    I[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    I[6] = c02 * id;
    I[7] = (A[1] * A[6] - A[0] * A[7]) * id;
    I[8] = (A[0] * A[4] - A[1] * A[3]) * id;
}

__device__ double det3(const double* A) {
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}

// Fit coefficients (eta, u0, sigma) -> paper parameters theta = (n', u',
// Theta'); invalid fits give theta = 0. One thread per cell.
__global__ void coef_to_theta_kernel(const double* coef, const int* status, int which, double* theta, long long ncell) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const double* k = coef + c * kCoef;
    double* th = theta + c * 10;
    for (int q = 0; q < 10; ++q) th[q] = 0.0;
    if (status[c * 2 + which] == 2) return;
    double m2[9] = {-2.0 * k[4], -k[5], -k[6], -k[5], -2.0 * k[7], -k[8], -k[6], -k[8], -2.0 * k[9]}, Thw[9];
    inv3(m2, Thw);
    double lam[3] = {k[1], k[2], k[3]}, uw[3], quad = 0.0;
    for (int p = 0; p < 3; ++p) {
        uw[p] = Thw[p * 3] * lam[0] + Thw[p * 3 + 1] * lam[1] + Thw[p * 3 + 2] * lam[2];
        quad += lam[p] * uw[p];
    }
    const double* u0 = k + 10;
    const double* sg = k + 13;
    th[0] = exp(k[0] + 0.5 * quad) * pow(2.0 * M_PI, 1.5) * sqrt(det3(Thw)) * sg[0] * sg[1] * sg[2];
    for (int p = 0; p < 3; ++p) th[1 + p] = u0[p] + sg[p] * uw[p];
    int q = 4;
    for (int p = 0; p < 3; ++p)
        for (int r = p; r < 3; ++r) th[q++] = sg[p] * sg[r] * Thw[p * 3 + r];
}

// ------------------------------------------------------------------ exchange

// Line parameters of one fitted Maxwellian for the exchange, from the fit
// coefficients (eta, u0, sigma): q(w) = eta0 + lambda.w + w^T mu w has its
// peak at w* = -mu^-1 lambda / 2 with value L = eta0 + lambda.w*/2, and
// w = w0 + h * index with h = dv/sigma, so in index space the exponent is
// L - 1/2 d^T P d with d = index - ic, ic = (w* - w0)/h, P = -2 H mu H.
// Along a v_z line (i, j fixed) this is
//   E(k) = Ec - hz (k - kc)^2,
//   Ec = L - 1/2 (Sxx dx^2 + 2 Sxy dx dy + Syy dy^2),  kc = icz + gx dx + gy dy,
// with (dx, dy) = (i, j) - (icx, icy), hz = Pzz/2, S = P_tt - p p^T / Pzz the
// Schur complement (p = (Pxz, Pyz)) and g = -p / Pzz.
// par[10] = (icx, icy, icz, Sxx, Sxy, Syy, gx, gy, hz, L); hz = 0 marks a fit
// that is not used.
constexpr int kPar = 10;

__device__ void maxwellian_line_params(const double* k, bool valid, const double* vmin, const double* dv, double* par) {
    for (int q = 0; q < kPar; ++q) par[q] = 0.0;
    if (!valid) return;
    double mu[9] = {k[4], 0.5 * k[5], 0.5 * k[6], 0.5 * k[5], k[7], 0.5 * k[8], 0.5 * k[6], 0.5 * k[8], k[9]};
    double mi[9];
    inv3(mu, mi);
    const double lam[3] = {k[1], k[2], k[3]};
    double ws[3], L = k[0], h[3], ic[3];
    for (int a = 0; a < 3; ++a) {
        ws[a] = -0.5 * (mi[a * 3] * lam[0] + mi[a * 3 + 1] * lam[1] + mi[a * 3 + 2] * lam[2]);
        L += 0.5 * lam[a] * ws[a];
    }
    const double* u0 = k + 10;
    const double* sg = k + 13;
    for (int a = 0; a < 3; ++a) {
        h[a] = dv[a] / sg[a];
        const double w0 = (vmin[a] + 0.5 * dv[a] - u0[a]) / sg[a];
        ic[a] = (ws[a] - w0) / h[a];
    }
    double P[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) P[a * 3 + b] = -2.0 * h[a] * h[b] * mu[a * 3 + b];
    const double pzz = P[8];
    if (!(pzz > 0.0) || !isfinite(L)) return;
    const double gx = -P[2] / pzz, gy = -P[5] / pzz;
    par[0] = ic[0];
    par[1] = ic[1];
    par[2] = ic[2];
    par[3] = P[0] + P[2] * gx;
    par[4] = P[1] + P[2] * gy;
    par[5] = P[4] + P[5] * gy;
    par[6] = gx;
    par[7] = gy;
    par[8] = 0.5 * pzz;
    par[9] = L;
}

// one thread per (cell, fit); the parameters are stored in the precision of
// f (T), packed [ncell][2][kPar] at the start of a.par
template <typename T>
__global__ void exchange_params_kernel(ExchangeArgs a) {
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g >= 2 * a.ncell) return;
    const long long cell = g >> 1;
    const int w = (int)(g & 1);
    const int stv = a.status[cell * 2], stf = a.status[cell * 2 + 1];
    const bool valid = stv != 2 && stf != 2;
    double par[kPar];
    maxwellian_line_params((w == 0 ? a.coef_v : a.coef_f) + cell * kCoef, valid, a.vmin, a.dv, par);
    T* out = reinterpret_cast<T*>(a.par) + cell * 2 * kPar + w * kPar;
#pragma unroll
    for (int q = 0; q < kPar; ++q) out[q] = (T)par[q];
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// r[k] += sgn * M(i, j, k) along the v_z line of this thread.
// FP32: per element, exponent in base 2 and ex2.approx (relative error
// about 2^-22).
template <int N>
__device__ __forceinline__ void add_maxwellian(float (&r)[N], const float* pd, int i, int j, float sgn,
                                               const double*) {
    const float hz = pd[8];
    if (!(hz > 0.f)) return;
    constexpr float kLog2e = 1.4426950408889634f;
    const float dx = (float)i - pd[0], dy = (float)j - pd[1];
    const float Q = pd[3] * dx * dx + 2.f * pd[4] * dx * dy + pd[5] * dy * dy;
    const float kc = pd[2] + pd[6] * dx + pd[7] * dy;
    const float Ec2 = (pd[9] - 0.5f * Q) * kLog2e;
    const float hz2 = hz * kLog2e;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const float tk = (float)k - kc;
        r[k] = fmaf(sgn, ex2_approx(fmaf(-hz2, tk * tk, Ec2)), r[k]);
    }
}

// FP64: M(k) = C A^m G(m) with k0 = floor(kc) (clamped to the line),
// m = k - k0, delta = kc - k0, C = exp(Ec - hz delta^2), A = exp(2 hz delta)
// and the per-cell table G(m) = exp(-hz m^2); three exponentials per line.
// The factors stay in range for hz <= 8 (sigma above a quarter cell);
// narrower Maxwellians take one exponential per element. Not inlined: with
// the line in registers and inlined twice into exchange_kernel<double, 20>,
// the optimised build gave wrong values (checked against a direct
// evaluation; the same code called out of line, every other block size and
// every optimisation level below -O2 agree with it), so the FP64 line update
// is a call.
template <int N>
__device__ __noinline__ void add_maxwellian(double (&r)[N], const double* pd, int i, int j, double sgn,
                                            const double* G) {
    const double hz = pd[8];
    if (!(hz > 0.0)) return;
    const double dx = i - pd[0], dy = j - pd[1];
    const double Q = pd[3] * dx * dx + 2.0 * pd[4] * dx * dy + pd[5] * dy * dy;
    const double kc = pd[2] + pd[6] * dx + pd[7] * dy;
    const double Ec = pd[9] - 0.5 * Q;
    if (hz > 8.0) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const double tk = k - kc;
            r[k] += sgn * exp(Ec - hz * tk * tk);
        }
        return;
    }
    double k0 = floor(kc);
    k0 = fmin(fmax(k0, 0.0), (double)(N - 1));
    const double delta = kc - k0;
    const double C = sgn * exp(Ec - hz * delta * delta);
    const double A = exp(2.0 * hz * delta);
    double Ap = exp(-2.0 * hz * delta * k0);
    const double* Gk = G + (N - 1) - (int)k0;  // Gk[k] = G(k - k0)
#pragma unroll
    for (int k = 0; k < N; ++k) {
        r[k] += C * (Ap * Gk[k]);
        Ap *= A;
    }
}

constexpr int ex_threads(int n) { return ((n * n + 31) / 32) * 32; }

// One CTA per cell at a time (persistent): thread t < N^2 owns the v_z line
// (i, j) = (t mod N, t / N), so each load and store of the block is a
// contiguous run of N^2 values. f <- f - M_V + M_F; if any value is negative
// all are clipped at zero and the cell rescaled to n_V (the limiter of
// Algorithm 1); cells whose fits are invalid are left alone. Fused with the
// moments of the new f.
template <typename T, int N>
__global__ void __launch_bounds__(ex_threads(N)) exchange_kernel(ExchangeArgs a) {
    __shared__ double red[20 * 32 + 20];
    __shared__ T ssum[32];
    __shared__ T sscale;
    __shared__ T spar[2 * kPar];
    __shared__ double gtab[2][sizeof(T) == 8 ? 2 * N - 1 : 1];
    T* f = reinterpret_cast<T*>(a.f);
    constexpr long long V = (long long)N * N * N;
    constexpr int NN = N * N;
    const int t = threadIdx.x;
    const int lane = t & 31, warp = t >> 5, nwarp = blockDim.x >> 5;
    const bool active = t < NN;
    const int i = active ? t % N : 0, j = active ? t / N : 0;
    const T* par = reinterpret_cast<const T*>(a.par);
    for (long long cell = blockIdx.x; cell < a.ncell; cell += gridDim.x) {
        T r[N];
        const T* src = f + cell * V + t;
        if (active) {
#pragma unroll
            for (int k = 0; k < N; ++k) r[k] = src[(long long)k * NN];
        }
        const int stv = a.status[cell * 2], stf = a.status[cell * 2 + 1];
        const bool skip = (stv == 2 || stf == 2);
        if (t < 2 * kPar) spar[t] = par[cell * 2 * kPar + t];
        if (sizeof(T) == 8 && t < 2 * (2 * N - 1)) {
            const int w = t / (2 * N - 1), m = t % (2 * N - 1) - (N - 1);
            const double hz = (double)par[cell * 2 * kPar + w * kPar + 8];
            gtab[w][sizeof(T) == 8 ? t % (2 * N - 1) : 0] = exp(-hz * (double)(m * m));
        }
        __syncthreads();
        int neg = 0;
        if (active && !skip) {
            add_maxwellian<N>(r, spar, i, j, T(-1), gtab[0]);
            add_maxwellian<N>(r, spar + kPar, i, j, T(1), gtab[1]);
            T mn = r[0];
#pragma unroll
            for (int k = 1; k < N; ++k) mn = fmin(mn, r[k]);
            neg = mn < T(0);
        }
        // any negative value in the block? (the clipped sums are only formed
        // in that rare case)
        const int anyneg = __syncthreads_or(neg);
        T scale = T(1);
        if (anyneg && !skip) {
            // per-warp sums of the clipped values in T, then FP64 across warps
            // on one thread for the rescale factor
            T ls = T(0);
            if (active) {
#pragma unroll
                for (int k = 0; k < N; ++k) ls += fmax(r[k], T(0));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) ls += __shfl_xor_sync(0xffffffffu, ls, o);
            if (lane == 0) ssum[warp] = ls;
            __syncthreads();
            if (t == 0) {
                double tot = 0.0;
                for (int w = 0; w < nwarp; ++w) tot += (double)ssum[w];
                const double vol = a.dv[0] * a.dv[1] * a.dv[2];
                const double nV = a.vmom[cell * 20];
                sscale = (T)(tot > 0.0 ? nV / (tot * vol) : 0.0);
                atomicAdd(&a.counters[CNT_CLIPPED], 1ull);
            }
            __syncthreads();
            scale = sscale;
        }
        T m[20];
#pragma unroll
        for (int q = 0; q < 20; ++q) m[q] = T(0);
        if (active) {
            T* dst = f + cell * V + t;
            const T c = T(0.5) * T(N - 1);
            T S0 = 0, S1 = 0, S2 = 0, S3 = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) {
                const T v = anyneg ? fmax(r[k], T(0)) * scale : r[k];
                if (!skip) dst[(long long)k * NN] = v;
                const T z = T(k) - c;
                const T v1 = v * z, v2 = v1 * z;
                S0 += v;
                S1 += v1;
                S2 += v2;
                S3 += v2 * z;
            }
            if (a.mom_out) line_products_z<T, N>(m, S0, S1, S2, S3, i, j);
        }
        if (a.mom_out) reduce_moments<T>(m, red, a.mom_out + cell * 20, a.conv);
        __syncthreads();
    }
}

// ------------------------------------------------------------------- 1D1V

// One warp per cell: 3-parameter fits (n, u, Theta) by Newton in FP64 on
// the natural parameters of exp(e0 + e1 w + e2 w^2), then the exchange. The
// lanes share the velocity cells of a moment evaluation; the sums are reduced
// by an xor butterfly, which leaves every lane with the same bits, so the
// Newton control flow is uniform over the warp.
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ int fit1d(const double* target, const FitArgs& a, double* theta, int* iters) {
    const int lane = threadIdx.x & 31;
    *iters = 0;
    const double n = target[0];
    theta[0] = theta[1] = theta[2] = 0.0;
    if (!(n > 0.0) || !isfinite(n)) return 2;
    const double u0 = target[1] / n, th0 = target[2] / n - u0 * u0;
    if (!(th0 > 0.0)) return 2;
    const double sg = sqrt(th0);
    const double w0 = (a.vmin[0] + 0.5 * a.dv[0] - u0) / sg, h = a.dv[0] / sg;
    double eta[3] = {log(n) - 0.5 * log(2.0 * M_PI) - 0.5 * log(th0), 0.0, -0.5};
    const double T[3] = {n, 0.0, n};
    auto eval = [&](const double* e, double* D, double* G4) {
        double p5[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int i = lane; i < a.nv; i += 32) {
            double w = w0 + i * h;
            double p = exp(e[0] + e[1] * w + e[2] * w * w) * a.dv[0];
            for (int q = 0; q < 5; ++q) {
                p5[q] += p;
                p *= w;
            }
        }
        for (int q = 0; q < 5; ++q) G4[q] = warp_sum_d(p5[q]);
        for (int q = 0; q < 3; ++q) D[q] = G4[q];
    };
    double D[3], G4[5];
    eval(eta, D, G4);
    bool conv = false;
    int it;
    for (it = 0; it <= a.max_iter; ++it) {
        double G[3], gmax = 0.0;
        bool fin = true;
        for (int q = 0; q < 3; ++q) {
            G[q] = D[q] - T[q];
            fin = fin && isfinite(G[q]);
            gmax = fmax(gmax, fabs(G[q]));
        }
        if (!fin) break;
        if (gmax <= a.tol * n) {
            conv = true;
            break;
        }
        if (it == a.max_iter) break;
        double J[9];
        for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q) J[p * 3 + q] = G4[p + q];
        double Ji[9], dl[3];
        inv3(J, Ji);
        for (int p = 0; p < 3; ++p) dl[p] = -(Ji[p * 3] * G[0] + Ji[p * 3 + 1] * G[1] + Ji[p * 3 + 2] * G[2]);
        double lam = 1.0, L0 = D[0], gd = 0.0, et[3];
        for (int q = 0; q < 3; ++q) {
            L0 -= eta[q] * T[q];
            gd += G[q] * dl[q];
        }
        for (int ls = 0; ls < 40; ++ls) {
            for (int q = 0; q < 3; ++q) et[q] = eta[q] + lam * dl[q];
            eval(et, D, G4);
            if (gmax <= 1e-6 * n) break;
            double L1 = D[0] - et[0] * T[0] - et[1] * T[1] - et[2] * T[2];
            if (isfinite(L1) && L1 <= L0 + 1e-4 * lam * gd) break;
            lam *= 0.5;
        }
        for (int q = 0; q < 3; ++q) eta[q] = et[q];
    }
    *iters = it;
    if (conv && eta[2] < 0.0) {
        double thw = -0.5 / eta[2], uw = thw * eta[1];
        theta[0] = exp(eta[0] + 0.5 * eta[1] * uw) * sqrt(2.0 * M_PI * thw) * sg;
        theta[1] = u0 + sg * uw;
        theta[2] = th0 * thw;
        return 0;
    }
    theta[0] = n;
    theta[1] = u0;
    theta[2] = th0;
    return 1;
}

__global__ void fit1d_kernel(FitArgs a) {
    const long long c = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    if (c >= a.ncell) return;  // whole warps leave together
    const bool lead = (threadIdx.x & 31) == 0;
    double tv[3] = {a.vmom[c * 4], a.vmom[c * 4 + 1], a.vmom[c * 4 + 2]};
    const double nF = a.fluid[c * 3];
    // non-finite or negative targets: a numeric error upstream (empty cells,
    // n = 0, are not)
    if (lead && a.numeric) {
        bool bad = !(tv[0] >= 0.0) || !(nF >= 0.0);
        for (int q = 0; q < 3; ++q) bad = bad || !isfinite(tv[q]) || !isfinite(a.fluid[c * 3 + q]);
        if (bad) *reinterpret_cast<volatile int*>(a.numeric) = VL_ENUMERIC;
    }
    const double scale = nF > 0.0 ? tv[0] / nF : 0.0;
    double tf[3];
    for (int q = 0; q < 3; ++q) tf[q] = a.fluid[c * 3 + q] * scale;
    double th[3];
    int itv, itf;
    int stv = fit1d(tv, a, th, &itv);
    if (lead)
        for (int q = 0; q < 3; ++q) a.coef_v[c * kCoef + q] = th[q];
    int stf = fit1d(tf, a, th, &itf);
    __syncwarp();  // every lane has read a.fluid before the lead lane rewrites it
    if (!lead) return;
    for (int q = 0; q < 3; ++q) {
        a.coef_f[c * kCoef + q] = th[q];
        a.fluid[c * 3 + q] = tf[q];
    }
    a.status[c * 2] = stv;
    a.status[c * 2 + 1] = stf;
    atomicAdd(&a.counters[CNT_ITERS], (unsigned long long)(itv + itf));
    unsigned long long fb = (stv == 1) + (stf == 1), inv = (stv == 2) + (stf == 2);
    if (fb) atomicAdd(&a.counters[CNT_FALLBACK], fb);
    if (inv) atomicAdd(&a.counters[CNT_INVALID], inv);
}

// One warp per cell, lanes over the velocity cells.
template <typename T>
__global__ void exchange1d_kernel(ExchangeArgs a) {
    const long long c = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    if (c >= a.ncell) return;  // whole warps leave together
    const int lane = threadIdx.x & 31;
    T* f = reinterpret_cast<T*>(a.f) + c * a.nv;
    const int stv = a.status[c * 2], stf = a.status[c * 2 + 1];
    if (stv != 2 && stf != 2) {
        const double* tv = a.coef_v + c * kCoef;
        const double* tf = a.coef_f + c * kCoef;
        bool neg = false;
        double sum = 0.0;
        for (int i = lane; i < a.nv; i += 32) {
            double v = a.vmin[0] + (i + 0.5) * a.dv[0];
            double mv = tv[0] / sqrt(2.0 * M_PI * tv[2]) * exp(-0.5 * (v - tv[1]) * (v - tv[1]) / tv[2]);
            double mf = tf[0] / sqrt(2.0 * M_PI * tf[2]) * exp(-0.5 * (v - tf[1]) * (v - tf[1]) / tf[2]);
            T x = (T)((double)f[i] - mv + mf);
            f[i] = x;
            neg |= x < T(0);
            sum += x > T(0) ? (double)x : 0.0;
        }
        if (__any_sync(0xffffffffu, neg)) {
            sum = warp_sum_d(sum);
            double sc = sum > 0.0 ? a.vmom[c * 4] / (sum * a.dv[0]) : 0.0;
            for (int i = lane; i < a.nv; i += 32) f[i] = (T)(f[i] > T(0) ? (double)f[i] * sc : 0.0);
            if (lane == 0) atomicAdd(&a.counters[CNT_CLIPPED], 1ull);
        }
    }
    if (a.mom_out) {
        double m[4] = {0, 0, 0, 0};
        for (int q = lane; q < a.nv; q += 32) {
            double v = a.vmin[0] + (q + 0.5) * a.dv[0], x = (double)f[q];
            m[0] += x; m[1] += v * x; m[2] += v * v * x; m[3] += v * v * v * x;
        }
        for (int p = 0; p < 4; ++p) m[p] = warp_sum_d(m[p]);
        if (lane == 0)
            for (int p = 0; p < 4; ++p) a.mom_out[c * 4 + p] = m[p] * a.dv[0];
    }
}

// ---------------------------------------------------------------- launchers

static int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 148;
    }
    return n;
}

// 1D1V: theta is stored directly in the coefficient slots
__global__ void theta1d_kernel(const double* coef, const int* status, int which, double* theta, long long ncell) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    for (int q = 0; q < 10; ++q) theta[c * 10 + q] = q < 3 && status[c * 2 + which] != 2 ? coef[c * kCoef + q] : 0.0;
}

cudaError_t launch_theta(const double* coef, const int* status, int which, double* theta, long long ncell, int nvdim,
                         cudaStream_t st) {
    unsigned grid = (unsigned)((ncell + 127) / 128);
    if (nvdim == 1) theta1d_kernel<<<grid, 128, 0, st>>>(coef, status, which, theta, ncell);
    else coef_to_theta_kernel<<<grid, 128, 0, st>>>(coef, status, which, theta, ncell);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_fit(const FitArgs& a, int nvdim, cudaStream_t st) {
    if (nvdim == 1) {
        unsigned grid = (unsigned)((a.ncell + 3) / 4);  // a warp per cell
        fit1d_kernel<<<grid, 128, 0, st>>>(a);
        count_launch();
        return cudaGetLastError();
    }
    return launch_newton3d(a, st);
}

template <typename T, int N>
static cudaError_t launch_exchange_n(const ExchangeArgs& a, cudaStream_t st) {
    {
        const long long n = 2 * a.ncell;
        exchange_params_kernel<T><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(a);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int threads = ex_threads(N);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, exchange_kernel<T, N>, threads, 0);
    if (per_sm < 1) per_sm = 1;
    long long grid = (long long)sm_count() * per_sm;
    if (grid > a.ncell) grid = a.ncell;
    exchange_kernel<T, N><<<(unsigned)grid, threads, 0, st>>>(a);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_exchange(const ExchangeArgs& a, int nvdim, int precision, cudaStream_t st) {
    if (nvdim == 1) {
        unsigned grid = (unsigned)((a.ncell + 3) / 4);  // a warp per cell
        if (precision == 64) exchange1d_kernel<double><<<grid, 128, 0, st>>>(a);
        else exchange1d_kernel<float><<<grid, 128, 0, st>>>(a);
        count_launch();
        return cudaGetLastError();
    }
#define VL_EX(T)                                                     \
    switch (a.nv) {                                                  \
        case 8: return launch_exchange_n<T, 8>(a, st);               \
        case 12: return launch_exchange_n<T, 12>(a, st);             \
        case 16: return launch_exchange_n<T, 16>(a, st);             \
        case 20: return launch_exchange_n<T, 20>(a, st);             \
        case 24: return launch_exchange_n<T, 24>(a, st);             \
        default: return cudaErrorInvalidValue;                       \
    }
    if (precision == 64) { VL_EX(double) }
    VL_EX(float)
#undef VL_EX
}

}  // namespace vl
