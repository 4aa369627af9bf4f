// Moment fitting (paper Sec. 2.2, Algorithm 1 "Moment Fitting").
//
// fit_kernel: one warp per spatial cell fits two discrete ten-moment
// Maxwellians, first to the moments of f (V) and then to the fluid moments
// rescaled by n_V / n_F (F). The fit makes the midpoint moments of degree <= 2
// of the sampled Maxwellian equal the targets, so that the exchange below
// changes the discrete moments of f by exactly (fluid - Vlasov). It is
// Newton's method on the natural parameters eta of
//     M(v) = exp(eta . phi(w)),  w_a = (v_a - u0_a) / sigma_a,
//     phi = (1, w_x, w_y, w_z, w_x^2, w_x w_y, w_x w_z, w_y^2, w_y w_z, w_z^2),
// with u0, sigma from the targets. The gradient (discrete moments minus
// targets) needs FP64 accuracy; on GB300 the FP64 pipe is ~1/58 of the FP32
// pipe, so the per-cell sums are evaluated in double-float arithmetic (pairs
// of floats with error-free transformations, ~44 significant bits) on the
// FP32 pipe, and FP64 is used only per cell and per line start:
//   * along a v_x line the exponent is quadratic in the cell index, so the
//     Maxwellian follows a two-term multiplicative recurrence (no exp per
//     cell); line starts follow the same recurrence across v_y lines;
//   * the Gram matrix sum M phi phi^T (the Jacobian) is summed in FP32 and
//     the 10x10 Newton system solved in FP32: the Newton step then carries a
//     ~1e-6 relative error, and each iteration still gains six digits;
//   * convergence is judged on the double-float/FP64 gradient: |D - T| <=
//     tol * n in the scaled coordinates w.
// Cells whose Maxwellian spans more than e^80 over the block (very cold or
// far off-grid), where a float recurrence could underflow, take a slow path
// with one FP64 exponential per cell.
//
// exchange_kernel: one CTA per cell: f <- f - f_M,V + f_M,F, clip negative
// values and rescale the cell to n_V (limiter of Algorithm 1), fused with the
// moments of the new f.
#include "common.cuh"
#include "kernels.cuh"

namespace vl {

enum { CNT_ITERS = 0, CNT_FALLBACK = 1, CNT_CLIPPED = 2, CNT_INVALID = 3 };
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

// float versions for the approximate per-cell setup
__device__ bool chol3f(const float* A) {
    float l00 = A[0];
    if (!(l00 > 0.f)) return false;
    l00 = sqrtf(l00);
    float l10 = A[3] / l00, l20 = A[6] / l00;
    float d1 = A[4] - l10 * l10;
    if (!(d1 > 0.f)) return false;
    float l11 = sqrtf(d1);
    float l21 = (A[7] - l20 * l10) / l11;
    float d2 = A[8] - l20 * l20 - l21 * l21;
    return d2 > 0.f;
}

__device__ void inv3f(const float* A, float* I) {
    float c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
    float id = 1.0f / (A[0] * c00 + A[1] * c01 + A[2] * c02);
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

// ------------------------------------------------------- double-float sums
// A value is hi + lo (two floats). Knuth's TwoSum and the FMA TwoProduct
// are error-free; products are left unnormalised (lo stays ~2^-24 hi).
struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_of(double x) {
    float h = (float)x;
    return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_val(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df df_mul(df a, df b) {
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return {p, e};
}

// running sum: s plus the accumulated error terms e
struct acc {
    float s, e;
};
__device__ __forceinline__ void acc_add(acc& A, float hi, float lo) {
    float s = A.s + hi;
    float bb = s - A.s;
    float err = (A.s - (s - bb)) + (hi - bb);
    A.s = s;
    A.e += err + lo;
}
// A += c * (hi + lo) for an exactly representable small constant c
__device__ __forceinline__ void acc_addc(acc& A, float hi, float lo, float c) {
    float p = hi * c;
    float e = fmaf(hi, c, -p);
    e = fmaf(lo, c, e);
    acc_add(A, p, e);
}

// ---------------------------------------------------------------- fitting

// Per-warp scratch in shared memory (keeps the register footprint of the
// element loops small).
struct WarpScratch {
    double kc[10];     // index-space exponent coefficients
    double et[10];     // trial parameters
    double eta0[10];   // starting parameters (fallback)
    float g[35];       // FP32 index moments of degree <= 4
    float W[35];       // the same in w-space
    float J[100];      // Gram matrix / its Cholesky factor
    float rhs[10], dl[10];
    float m[20];       // double-float index moments of degree <= 2 (hi, lo)
    double eta[10];    // current parameters
    double tgt[10];    // targets of the current fit
    double coef[16];   // result of the current fit
    double wc[3], h[3], u0[3], sg[3];
    float shift[3];    // moment weights use c - shift (origin near the mass)
    double Jd[100];    // FP64 Gram matrix of the precise mode
    double dd[10];     // FP64 Newton step of the precise mode
};

// Index-space coefficients of the exponent, with centred indices
// c_a = i_a - (N-1)/2: q = k0 + sum_a k_a c_a + sum_{a<=b} k_ab c_a c_b,
// stored as kc = (k0, kx, ky, kz, kxx, kxy, kxz, kyy, kyz, kzz).
// Lane t < 10 computes kc[t] from eta and the scaled grid (wc at the box
// centre, h = dv / sigma).
__device__ void index_coefficients(const double* eta, const double* wc, const double* h, double* kc) {
    const int lane = threadIdx.x & 31;
    // eta: 0:1 1:x 2:y 3:z 4:xx 5:xy 6:xz 7:yy 8:yz 9:zz
    const double e0 = eta[0], ex = eta[1], ey = eta[2], ez = eta[3];
    const double exx = eta[4], exy = eta[5], exz = eta[6], eyy = eta[7], eyz = eta[8], ezz = eta[9];
    double v = 0.0;
    switch (lane) {
        case 0:
            v = e0 + ex * wc[0] + ey * wc[1] + ez * wc[2] + exx * wc[0] * wc[0] + exy * wc[0] * wc[1] +
                exz * wc[0] * wc[2] + eyy * wc[1] * wc[1] + eyz * wc[1] * wc[2] + ezz * wc[2] * wc[2];
            break;
        case 1: v = h[0] * (ex + 2.0 * exx * wc[0] + exy * wc[1] + exz * wc[2]); break;
        case 2: v = h[1] * (ey + 2.0 * eyy * wc[1] + exy * wc[0] + eyz * wc[2]); break;
        case 3: v = h[2] * (ez + 2.0 * ezz * wc[2] + exz * wc[0] + eyz * wc[1]); break;
        case 4: v = exx * h[0] * h[0]; break;
        case 5: v = exy * h[0] * h[1]; break;
        case 6: v = exz * h[0] * h[2]; break;
        case 7: v = eyy * h[1] * h[1]; break;
        case 8: v = eyz * h[1] * h[2]; break;
        case 9: v = ezz * h[2] * h[2]; break;
        default: break;
    }
    if (lane < 10) kc[lane] = v;
    __syncwarp();
}

// monomial c_x^p c_y^q c_z^r with p+q+r <= 4 -> index in [0, 35)
__host__ __device__ constexpr int mono4(int p, int q, int r) {
    int d = p + q + r, idx = 0;
    for (int e = 0; e < d; ++e) idx += (e + 1) * (e + 2) / 2;
    for (int pp = d; pp > p; --pp) idx += d - pp + 1;
    return idx + (d - p) - q;
}

// warp reduction of a double-float accumulator (result broadcast from lane 0)
__device__ __forceinline__ df reduce_acc(acc a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float s = __shfl_xor_sync(0xffffffffu, a.s, o);
        float e = __shfl_xor_sync(0xffffffffu, a.e, o);
        acc_add(a, s, e);
    }
    return {bcastf(a.s, 0), bcastf(a.e, 0)};
}

__device__ __forceinline__ float reduce_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return bcastf(v, 0);
}

// per-line index moments -> cell accumulators
__device__ __forceinline__ void line_to_cell(acc* m, acc S0, acc S1, acc S2, float cj, float ck) {
    acc_add(m[0], S0.s, S0.e);
    acc_add(m[1], S1.s, S1.e);
    acc_addc(m[2], S0.s, S0.e, cj);
    acc_addc(m[3], S0.s, S0.e, ck);
    acc_add(m[4], S2.s, S2.e);
    acc_addc(m[5], S1.s, S1.e, cj);
    acc_addc(m[6], S1.s, S1.e, ck);
    acc_addc(m[7], S0.s, S0.e, cj * cj);
    acc_addc(m[8], S0.s, S0.e, cj * ck);
    acc_addc(m[9], S0.s, S0.e, ck * ck);
}

__device__ __forceinline__ void gram_line(float* g, const float* T, float cj, float ck) {
    float pj[5], pk[5];
    pj[0] = pk[0] = 1.f;
#pragma unroll
    for (int q = 1; q < 5; ++q) {
        pj[q] = pj[q - 1] * cj;
        pk[q] = pk[q - 1] * ck;
    }
#pragma unroll
    for (int p = 0; p <= 4; ++p)
#pragma unroll
        for (int q = 0; q <= 4 - p; ++q)
#pragma unroll
            for (int r = 0; r <= 4 - p - q; ++r) g[mono4(p, q, r)] = fmaf(T[p], pj[q] * pk[r], g[mono4(p, q, r)]);
}

// Can the float recurrences represent every value and step over the block?
// (the minimum of a concave quadratic over a box is at a corner; one-cell
// steps are linear in position, extreme at the corners)
template <int N>
__device__ bool fast_ok(const double* kcd) {
    const int lane = threadIdx.x & 31;
    constexpr float hN = 0.5f * (N - 1);
    const float k0 = (float)kcd[0], kx = (float)kcd[1], ky = (float)kcd[2], kz = (float)kcd[3];
    const float kxx = (float)kcd[4], kxy = (float)kcd[5], kxz = (float)kcd[6], kyy = (float)kcd[7],
                kyz = (float)kcd[8], kzz = (float)kcd[9];
    bool ok = kcd[4] < 0.0;
    if (lane < 8) {
        float x = (lane & 1) ? hN : -hN, y = (lane & 2) ? hN : -hN, z = (lane & 4) ? hN : -hN;
        float q = k0 + kx * x + ky * y + kz * z + kxx * x * x + kxy * x * y + kxz * x * z + kyy * y * y + kyz * y * z +
                  kzz * z * z;
        ok = ok && (q > -80.f) && (q < 80.f);
    } else if (lane < 16) {
        float y = (lane & 1) ? hN : -hN, z = (lane & 2) ? hN : -hN, x = (lane & 4) ? hN - 1.f : -hN;
        float d = kxx * (2.f * x + 1.f) + kx + kxy * y + kxz * z;
        ok = ok && fabsf(d) < 80.f;
    } else if (lane < 24) {
        float z = (lane & 1) ? hN : -hN, y = (lane & 2) ? hN - 1.f : -hN;
        float d = kyy * (2.f * y + 1.f) + ky - hN * kxy + kyz * z;
        ok = ok && fabsf(d) < 80.f && fabsf(2.f * kxx) < 80.f && fabsf(2.f * kyy) < 80.f && fabsf(kxy) < 80.f;
    }
    return __all_sync(0xffffffffu, ok);
}

// Fast path: double-float recurrences for the index moments of degree <= 2
// (into ws.m) and, if wanted, FP32 recurrences for degree <= 4 (ws.g).
template <int N>
__device__ void eval_fast(WarpScratch& ws, bool want_gram) {
    const int lane = threadIdx.x & 31;
    constexpr float hN = 0.5f * (N - 1);
    const double* kc = ws.kc;
    // per-cell ratios: inner exp(2 kxx), line-to-line exp(2 kyy), exp(kxy)
    const double arg = lane == 0 ? 2.0 * kc[4] : (lane == 1 ? 2.0 * kc[7] : kc[5]);
    const double ev = lane < 3 ? exp(arg) : 0.0;
    const double e_in = bcast(ev, 0), e_j = bcast(ev, 1), e_xy = bcast(ev, 2);
    constexpr int R = (N * N + 31) / 32;
    const int l0 = lane * R;
    const int l1 = min(N * N, l0 + R);
    const float shx = ws.shift[0], shy = ws.shift[1], shz = ws.shift[2];
    {
        const df rho_in = df_of(e_in), rho_j = df_of(e_j), exy = df_of(e_xy);
        acc m[10];
#pragma unroll
        for (int q = 0; q < 10; ++q) m[q] = {0.f, 0.f};
        df Ms = {0.f, 0.f}, rs = {0.f, 0.f}, rl = {0.f, 0.f};
#pragma unroll 1
        for (int l = l0; l < l1; ++l) {
            const int j = l % N, k = l / N;
            const float cj = (float)j - hN, ck = (float)k - hN;
            if (l == l0 || j == 0) {
                const double B = kc[1] + kc[5] * cj + kc[6] * ck;
                const double C = kc[0] + kc[2] * cj + kc[3] * ck + kc[7] * cj * cj + kc[8] * cj * ck + kc[9] * ck * ck;
                Ms = df_of(exp(kc[4] * hN * hN - B * hN + C));
                rs = df_of(exp(kc[4] * (2.0 - N) + B));
                rl = df_of(exp(kc[2] - hN * kc[5] + kc[7] * (2.0 * cj + 1.0) + kc[8] * ck));
            }
            acc S0 = {0.f, 0.f}, S1 = {0.f, 0.f}, S2 = {0.f, 0.f};
            df M = Ms, r = rs;
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const float ci = ((float)i - hN) - shx;
                acc_add(S0, M.hi, M.lo);
                acc_addc(S1, M.hi, M.lo, ci);
                acc_addc(S2, M.hi, M.lo, ci * ci);
                M = df_mul(M, r);
                r = df_mul(r, rho_in);
            }
            line_to_cell(m, S0, S1, S2, cj - shy, ck - shz);
            Ms = df_mul(Ms, rl);
            rl = df_mul(rl, rho_j);
            rs = df_mul(rs, exy);
        }
#pragma unroll
        for (int q = 0; q < 10; ++q) {
            df v = reduce_acc(m[q]);
            if (lane == 0) {
                ws.m[2 * q] = v.hi;
                ws.m[2 * q + 1] = v.lo;
            }
        }
    }
    if (want_gram) {
        float g[35];
#pragma unroll
        for (int q = 0; q < 35; ++q) g[q] = 0.f;
        const float rin = (float)e_in, rj = (float)e_j, rxy = (float)e_xy;
        float ms = 0.f, r0 = 0.f, rls = 0.f;
#pragma unroll 1
        for (int l = l0; l < l1; ++l) {
            const int j = l % N, k = l / N;
            const float cj = (float)j - hN, ck = (float)k - hN;
            if (l == l0 || j == 0) {
                const float kxx = (float)kc[4], kxy = (float)kc[5];
                const float B = (float)kc[1] + kxy * cj + (float)kc[6] * ck;
                const float C = (float)kc[0] + (float)kc[2] * cj + (float)kc[3] * ck + (float)kc[7] * cj * cj +
                                (float)kc[8] * cj * ck + (float)kc[9] * ck * ck;
                ms = expf(kxx * hN * hN - B * hN + C);
                r0 = expf(kxx * (2.f - N) + B);
                rls = expf((float)kc[2] - hN * kxy + (float)kc[7] * (2.f * cj + 1.f) + (float)kc[8] * ck);
            }
            float T[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
            float M = ms, r = r0;
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const float ci = ((float)i - hN) - shx, c2 = ci * ci;
                T[0] += M;
                T[1] = fmaf(M, ci, T[1]);
                T[2] = fmaf(M, c2, T[2]);
                T[3] = fmaf(M, c2 * ci, T[3]);
                T[4] = fmaf(M, c2 * c2, T[4]);
                M *= r;
                r *= rin;
            }
            gram_line(g, T, cj - shy, ck - shz);
            ms *= rls;
            rls *= rj;
            r0 *= rxy;
        }
#pragma unroll
        for (int q = 0; q < 35; ++q) {
            float v = reduce_f(g[q]);
            if (lane == 0) ws.g[q] = v;
        }
    }
    __syncwarp();
}

// Slow path: one FP64 exponential per cell (any exponent range).
template <int N>
__device__ void eval_slow(WarpScratch& ws, bool want_gram) {
    const int lane = threadIdx.x & 31;
    constexpr double hN = 0.5 * (N - 1);
    const double* kc = ws.kc;
    double m[10];
    float g[35];
#pragma unroll
    for (int q = 0; q < 10; ++q) m[q] = 0.0;
#pragma unroll
    for (int q = 0; q < 35; ++q) g[q] = 0.f;
#pragma unroll 1
    for (int l = lane; l < N * N; l += 32) {
        const int j = l % N, k = l / N;
        const double cj = j - hN, ck = k - hN;
        const double B = kc[1] + kc[5] * cj + kc[6] * ck;
        const double C = kc[0] + kc[2] * cj + kc[3] * ck + kc[7] * cj * cj + kc[8] * cj * ck + kc[9] * ck * ck;
        double S0 = 0, S1 = 0, S2 = 0;
        float T[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        const double shx = ws.shift[0];
#pragma unroll 1
        for (int i = 0; i < N; ++i) {
            const double cq = i - hN;
            const double M = exp(C + cq * (B + kc[4] * cq));
            const double ci = cq - shx;
            S0 += M;
            S1 = fma(M, ci, S1);
            S2 = fma(M, ci * ci, S2);
            if (want_gram) {
                float Mf = (float)M, cf = (float)ci;
                T[0] += Mf;
                T[1] = fmaf(Mf, cf, T[1]);
                T[2] = fmaf(Mf, cf * cf, T[2]);
                T[3] = fmaf(Mf, cf * cf * cf, T[3]);
                T[4] = fmaf(Mf, cf * cf * cf * cf, T[4]);
            }
        }
        const double sj = cj - ws.shift[1], sk = ck - ws.shift[2];
        m[0] += S0; m[1] += S1; m[2] += sj * S0; m[3] += sk * S0; m[4] += S2;
        m[5] += sj * S1; m[6] += sk * S1; m[7] += sj * sj * S0; m[8] += sj * sk * S0; m[9] += sk * sk * S0;
        if (want_gram) gram_line(g, T, (float)sj, (float)sk);
    }
#pragma unroll
    for (int q = 0; q < 10; ++q) {
        df v = df_of(warp_sum(m[q]));
        if (lane == 0) {
            ws.m[2 * q] = v.hi;
            ws.m[2 * q + 1] = v.lo;
        }
    }
    if (want_gram)
#pragma unroll
        for (int q = 0; q < 35; ++q) {
            float v = reduce_f(g[q]);
            if (lane == 0) ws.g[q] = v;
        }
    __syncwarp();
}

// w-space discrete moment D_t (lane t < 10) from the index moments:
// w_a = wc_a + h_a c_a, times the cell volume.
__device__ double w_moment(int t, const float* mf, const double* wc, const double* h, double vol) {
    auto M = [&](int q) { return (double)mf[2 * q] + (double)mf[2 * q + 1]; };
    const double m0 = M(0);
    switch (t) {
        case 0: return vol * m0;
        case 1: return vol * (wc[0] * m0 + h[0] * M(1));
        case 2: return vol * (wc[1] * m0 + h[1] * M(2));
        case 3: return vol * (wc[2] * m0 + h[2] * M(3));
        case 4: return vol * (wc[0] * wc[0] * m0 + 2.0 * wc[0] * h[0] * M(1) + h[0] * h[0] * M(4));
        case 5: return vol * (wc[0] * wc[1] * m0 + wc[0] * h[1] * M(2) + h[0] * wc[1] * M(1) + h[0] * h[1] * M(5));
        case 6: return vol * (wc[0] * wc[2] * m0 + wc[0] * h[2] * M(3) + h[0] * wc[2] * M(1) + h[0] * h[2] * M(6));
        case 7: return vol * (wc[1] * wc[1] * m0 + 2.0 * wc[1] * h[1] * M(2) + h[1] * h[1] * M(7));
        case 8: return vol * (wc[1] * wc[2] * m0 + wc[1] * h[2] * M(3) + h[1] * wc[2] * M(2) + h[1] * h[2] * M(8));
        case 9: return vol * (wc[2] * wc[2] * m0 + 2.0 * wc[2] * h[2] * M(3) + h[2] * h[2] * M(9));
        default: return 0.0;
    }
}

// Gram matrix J = sum M phi phi^T dv^3 in w-space (FP32) from the index
// moments of degree <= 4 (binomial expansion per axis); lanes share the 35
// w-space moments, lane 0 assembles J.
__device__ void gram_matrix(WarpScratch& ws, const double* wcd, const double* hd, float vol) {
    const int lane = threadIdx.x & 31;
    const float wc[3] = {(float)wcd[0], (float)wcd[1], (float)wcd[2]};
    const float h[3] = {(float)hd[0], (float)hd[1], (float)hd[2]};
    const float binom[5][5] = {{1, 0, 0, 0, 0}, {1, 1, 0, 0, 0}, {1, 2, 1, 0, 0}, {1, 3, 3, 1, 0}, {1, 4, 6, 4, 1}};
    for (int t = lane; t < 35; t += 32) {
        // decode t -> (A, B, C)
        int A = 0, B = 0, C = 0;
        for (int a = 0; a <= 4; ++a)
            for (int b = 0; b <= 4 - a; ++b)
                for (int c = 0; c <= 4 - a - b; ++c)
                    if (mono4(a, b, c) == t) {
                        A = a;
                        B = b;
                        C = c;
                    }
        float s = 0.f;
        for (int p = 0; p <= A; ++p)
            for (int q = 0; q <= B; ++q)
                for (int r = 0; r <= C; ++r) {
                    float w = binom[A][p] * binom[B][q] * binom[C][r];
                    for (int u = 0; u < A - p; ++u) w *= wc[0];
                    for (int u = 0; u < p; ++u) w *= h[0];
                    for (int u = 0; u < B - q; ++u) w *= wc[1];
                    for (int u = 0; u < q; ++u) w *= h[1];
                    for (int u = 0; u < C - r; ++u) w *= wc[2];
                    for (int u = 0; u < r; ++u) w *= h[2];
                    s = fmaf(w, ws.g[mono4(p, q, r)], s);
                }
        ws.W[t] = s * vol;
    }
    __syncwarp();
    const int E[10][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0},
                          {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2}};
    for (int e = lane; e < 100; e += 32) {
        int a = e / 10, b = e % 10;
        ws.J[e] = ws.W[mono4(E[a][0] + E[b][0], E[a][1] + E[b][1], E[a][2] + E[b][2])];
    }
    __syncwarp();
}

// Cholesky solve of the SPD 10x10 system J x = rhs in FP32 by lane 0
// (writes ws.dl); returns the success flag on all lanes.
__device__ bool solve10f(WarpScratch& ws) {
    const int lane = threadIdx.x & 31;
    int ok = 1;
    if (lane == 0) {
        float* J = ws.J;
        for (int i = 0; i < 10 && ok; ++i)
            for (int j = 0; j <= i; ++j) {
                float s = J[i * 10 + j];
                for (int k = 0; k < j; ++k) s -= J[i * 10 + k] * J[j * 10 + k];
                if (i == j) {
                    if (!(s > 0.f)) {
                        ok = 0;
                        break;
                    }
                    J[i * 10 + i] = sqrtf(s);
                } else {
                    J[i * 10 + j] = s / J[j * 10 + j];
                }
            }
        if (ok) {
            float y[10];
            for (int i = 0; i < 10; ++i) {
                float s = ws.rhs[i];
                for (int k = 0; k < i; ++k) s -= J[i * 10 + k] * y[k];
                y[i] = s / J[i * 10 + i];
            }
            for (int i = 9; i >= 0; --i) {
                float s = y[i];
                for (int k = i + 1; k < 10; ++k) s -= J[k * 10 + i] * ws.dl[k];
                ws.dl[i] = s / J[i * 10 + i];
            }
        }
    }
    __syncwarp();
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// Precise mode (cells where the FP32 Jacobian does not converge within a
// few iterations, e.g. Maxwellians truncated by the velocity box): the Gram
// matrix in FP64 with one exponential per cell, solved in FP64 by lane 0.
template <int N>
__device__ bool precise_step(WarpScratch& ws, const double* wc, const double* h, double vol, double Gl) {
    const int lane = threadIdx.x & 31;
    constexpr double hN = 0.5 * (N - 1);
    const double* kc = ws.kc;
    double W[35];
#pragma unroll
    for (int q = 0; q < 35; ++q) W[q] = 0.0;
#pragma unroll 1
    for (int l = lane; l < N * N; l += 32) {
        const int j = l % N, k = l / N;
        const double cj = j - hN, ck = k - hN;
        const double B = kc[1] + kc[5] * cj + kc[6] * ck;
        const double C = kc[0] + kc[2] * cj + kc[3] * ck + kc[7] * cj * cj + kc[8] * cj * ck + kc[9] * ck * ck;
        double T[5] = {0, 0, 0, 0, 0};
#pragma unroll 1
        for (int i = 0; i < N; ++i) {
            const double ci = i - hN;
            const double M = exp(C + ci * (B + kc[4] * ci));
            const double w = wc[0] + h[0] * ci;
            double p = M;
            for (int q = 0; q < 5; ++q) {
                T[q] += p;
                p *= w;
            }
        }
        const double wy = wc[1] + h[1] * cj, wz = wc[2] + h[2] * ck;
        double py[5], pz[5];
        py[0] = pz[0] = 1.0;
        for (int q = 1; q < 5; ++q) {
            py[q] = py[q - 1] * wy;
            pz[q] = pz[q - 1] * wz;
        }
        for (int a = 0; a <= 4; ++a)
            for (int b = 0; b <= 4 - a; ++b)
                for (int c = 0; c <= 4 - a - b; ++c) W[mono4(a, b, c)] += T[a] * py[b] * pz[c];
    }
#pragma unroll
    for (int q = 0; q < 35; ++q) W[q] = warp_sum(W[q]) * vol;
    const int E[10][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0},
                          {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2}};
    double rhs = -Gl;
    double g[10];
    for (int q = 0; q < 10; ++q) g[q] = bcast(rhs, q);
    int ok = 1;
    if (lane == 0) {
        double* J = ws.Jd;
        for (int e = 0; e < 100; ++e) {
            int a = e / 10, b = e % 10;
            J[e] = W[mono4(E[a][0] + E[b][0], E[a][1] + E[b][1], E[a][2] + E[b][2])];
        }
        for (int i = 0; i < 10 && ok; ++i)
            for (int j = 0; j <= i; ++j) {
                double s = J[i * 10 + j];
                for (int k = 0; k < j; ++k) s -= J[i * 10 + k] * J[j * 10 + k];
                if (i == j) {
                    if (!(s > 0.0)) {
                        ok = 0;
                        break;
                    }
                    J[i * 10 + i] = sqrt(s);
                } else {
                    J[i * 10 + j] = s / J[j * 10 + j];
                }
            }
        if (ok) {
            double y[10];
            for (int i = 0; i < 10; ++i) {
                double s = g[i];
                for (int k = 0; k < i; ++k) s -= J[i * 10 + k] * y[k];
                y[i] = s / J[i * 10 + i];
            }
            for (int i = 9; i >= 0; --i) {
                double s = y[i];
                for (int k = i + 1; k < 10; ++k) s -= J[k * 10 + i] * ws.dd[k];
                ws.dd[i] = s / J[i * 10 + i];
            }
        }
    }
    __syncwarp();
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

template <int N>
__device__ __forceinline__ void evaluate(WarpScratch& ws, const double* eta, const double* wc, const double* h,
                                         bool gram) {
    index_coefficients(eta, wc, h, ws.kc);
    if (fast_ok<N>(ws.kc)) eval_fast<N>(ws, gram);
    else eval_slow<N>(ws, gram);
}

// One fit; all lanes of the warp call it with the same target. Writes the
// coefficients (eta, u0, sigma) of the fitted or fallback Maxwellian.
// Returns status 0 converged, 1 fallback, 2 invalid targets.
template <int N>
__device__ int fit_one(WarpScratch& ws, const FitArgs& a, int* iters) {
    const int lane = threadIdx.x & 31;
    const double* t = ws.tgt;
    *iters = 0;
    const double n = t[0];
    if (lane < kCoef) ws.coef[lane] = 0.0;
    __syncwarp();
    if (!(n > 0.0) || !isfinite(n)) return 2;
    // scaled coordinates from FP32 estimates (any u0, sigma define a valid
    // change of variables; the targets T below are transformed exactly)
    const float nf = (float)n;
    {
        float u0f[3], Th[9];
        for (int q = 0; q < 3; ++q) u0f[q] = (float)t[1 + q] / nf;
        const int pk[3][3] = {{4, 5, 6}, {5, 7, 8}, {6, 8, 9}};
        for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q) Th[p * 3 + q] = (float)t[pk[p][q]] / nf - u0f[p] * u0f[q];
        if (!chol3f(Th)) return 2;
        if (lane < 3) {
            const int q = lane;
            ws.u0[q] = (double)u0f[q];
            ws.sg[q] = (double)sqrtf(Th[q * 4]);
            ws.h[q] = a.dv[q] / ws.sg[q];
            ws.wc[q] = (a.vmin[q] + 0.5 * N * a.dv[q] - ws.u0[q]) / ws.sg[q];
            // integer cell nearest to the mean: origin of the moment weights
            float ic = rintf((float)((ws.u0[q] - a.vmin[q]) / a.dv[q] - 0.5));
            ic = fminf(fmaxf(ic, 0.f), (float)(N - 1));
            ws.shift[q] = ic - 0.5f * (N - 1);
        }
        __syncwarp();
    }
    // w at the origin of the moment weights
    double wm[3];
    for (int q = 0; q < 3; ++q) wm[q] = ws.wc[q] + ws.h[q] * (double)ws.shift[q];
    const double vol = a.dv[0] * a.dv[1] * a.dv[2];
    // targets in w-space, lane t < 10 holds T_t
    double Tl = 0.0;
    {
        const int pk[3][3] = {{4, 5, 6}, {5, 7, 8}, {6, 8, 9}};
        const int ab[10][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
        const double* u0 = ws.u0;
        const double* sg = ws.sg;
        if (lane == 0) Tl = n;
        else if (lane < 4) {
            int p = lane - 1;
            Tl = (t[1 + p] - n * u0[p]) / sg[p];
        } else if (lane < 10) {
            int p = ab[lane][0], q = ab[lane][1];
            Tl = (t[pk[p][q]] - u0[p] * t[1 + q] - u0[q] * t[1 + p] + n * u0[p] * u0[q]) / (sg[p] * sg[q]);
        }
    }
    // start: continuous Maxwellian of the targets in w-space (FP32 estimate)
    {
        float Cw[9], P[9], mw[3];
        for (int p = 0; p < 3; ++p) mw[p] = (float)(bcast(Tl, 1 + p) / n);
        const int sidx[3][3] = {{4, 5, 6}, {5, 7, 8}, {6, 8, 9}};
        for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q) Cw[p * 3 + q] = (float)(bcast(Tl, sidx[p][q]) / n) - mw[p] * mw[q];
        inv3f(Cw, P);
        float detC = Cw[0] * (Cw[4] * Cw[8] - Cw[5] * Cw[7]) - Cw[1] * (Cw[3] * Cw[8] - Cw[5] * Cw[6]) +
                     Cw[2] * (Cw[3] * Cw[7] - Cw[4] * Cw[6]);
        float lam[3], quad = 0.f;
        for (int p = 0; p < 3; ++p) lam[p] = P[p * 3] * mw[0] + P[p * 3 + 1] * mw[1] + P[p * 3 + 2] * mw[2];
        for (int p = 0; p < 3; ++p) quad += mw[p] * lam[p];
        // M(v) = n (2 pi)^-3/2 det(Theta)^-1/2 exp(...), Theta = S Cw S
        float logdet = logf(detC) + 2.f * logf((float)(ws.sg[0] * ws.sg[1] * ws.sg[2]));
        const float init[10] = {logf(nf) - 1.5f * logf(6.2831853f) - 0.5f * logdet - 0.5f * quad,
                                lam[0], lam[1], lam[2], -0.5f * P[0], -P[1], -P[2], -0.5f * P[4], -P[5], -0.5f * P[8]};
        if (lane < 10) {
            float v = 0.f;
#pragma unroll
            for (int q = 0; q < 10; ++q)
                if (q == lane) v = init[q];
            ws.eta[lane] = v;
            ws.eta0[lane] = v;
        }
        __syncwarp();
    }

    bool converged = false;
    int it = 0;
    evaluate<N>(ws, ws.eta, ws.wc, ws.h, true);
    bool have_gram = true;
    for (it = 0; it <= a.max_iter; ++it) {
        const double Dl = lane < 10 ? w_moment(lane, ws.m, wm, ws.h, vol) : 0.0;
        const double Gl = Dl - Tl;
        if (!__all_sync(0xffffffffu, isfinite(Gl))) break;
        if (__all_sync(0xffffffffu, fabs(Gl) <= a.tol * n)) {
            converged = true;
            break;
        }
        if (it == a.max_iter) break;
        float gmax = fabsf((float)(Gl / n));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) gmax = fmaxf(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
        gmax = bcastf(gmax, 0);
        const bool precise = it >= 6;
        if (precise) {
            // FP64 Jacobian at this point (kc of the current parameters)
            index_coefficients(ws.eta, ws.wc, ws.h, ws.kc);
            if (!precise_step<N>(ws, ws.wc, ws.h, vol, Gl)) break;
            if (lane < 10) ws.dl[lane] = (float)0.0;
            __syncwarp();
        } else {
            if (!have_gram) {
                evaluate<N>(ws, ws.eta, ws.wc, ws.h, true);  // refresh the Jacobian at this point
                have_gram = true;
            }
            gram_matrix(ws, wm, ws.h, (float)vol);
            if (lane < 10) ws.rhs[lane] = -(float)Gl;
            __syncwarp();
            if (!solve10f(ws)) break;
            if (lane < 10) ws.dd[lane] = (double)ws.dl[lane];
            __syncwarp();
        }
        // damped step: backtracking on L(eta) = D_0 - eta . T while far away
        const bool damp = gmax > 1e-6f;
        double L0 = 0.0, gd = 0.0;
        if (damp) {
            L0 = bcast(Dl, 0) - warp_sum(lane < 10 ? ws.eta[lane] * Tl : 0.0);
            gd = warp_sum(lane < 10 ? Gl * ws.dd[lane] : 0.0);
        }
        double lamb = 1.0;
        const bool gram_next = gmax > 1e-7f;
        for (int ls = 0; ls < 40; ++ls) {
            if (lane < 10) ws.et[lane] = ws.eta[lane] + lamb * ws.dd[lane];
            __syncwarp();
            evaluate<N>(ws, ws.et, ws.wc, ws.h, gram_next);
            if (!damp) break;
            const double D0 = vol * ((double)ws.m[0] + (double)ws.m[1]);
            const double L1 = D0 - warp_sum(lane < 10 ? ws.et[lane] * Tl : 0.0);
            if (isfinite(L1) && L1 <= L0 + 1e-4 * lamb * gd) break;
            lamb *= 0.5;
        }
        have_gram = gram_next;
        if (lane < 10) ws.eta[lane] = ws.et[lane];
        __syncwarp();
    }
    *iters = it;
    bool pd = false;
    if (converged) {
        // the fitted exponent must be a Gaussian: -2 mu positive definite
        const double* e = ws.eta;
        double m2[9] = {-2.0 * e[4], -e[5], -e[6], -e[5], -2.0 * e[7], -e[8], -e[6], -e[8], -2.0 * e[9]}, L[9];
        pd = chol3(m2, L);
    }
    const bool good = converged && pd;
    if (lane < 10) ws.coef[lane] = good ? ws.eta[lane] : ws.eta0[lane];
    else if (lane < 13) ws.coef[lane] = ws.u0[lane - 10];
    else if (lane < 16) ws.coef[lane] = ws.sg[lane - 13];
    __syncwarp();
    return good ? 0 : 1;
}

template <int N>
__global__ void __launch_bounds__(128) fit_kernel(FitArgs a) {
    __shared__ WarpScratch scratch[4];
    const int lane = threadIdx.x & 31;
    WarpScratch& ws = scratch[threadIdx.x >> 5];
    const long long wpb = blockDim.x >> 5;
    const long long warp0 = blockIdx.x * wpb + (threadIdx.x >> 5);
    for (long long cell = warp0; cell < a.ncell; cell += (long long)gridDim.x * wpb) {
        // V targets: the moments of f
        if (lane < 10) ws.tgt[lane] = a.vmom[cell * 20 + lane];
        __syncwarp();
        const double nV = ws.tgt[0];
        int itv, itf;
        int stv = fit_one<N>(ws, a, &itv);
        if (lane < kCoef) a.coef_v[cell * kCoef + lane] = ws.coef[lane];
        __syncwarp();
        // F targets: the fluid moments rescaled by n_V / n_F
        const double nF = a.fluid[cell * 10];
        const double scale = nF > 0.0 ? nV / nF : 0.0;
        if (lane < 10) {
            double v = a.fluid[cell * 10 + lane] * scale;
            ws.tgt[lane] = v;
            a.fluid[cell * 10 + lane] = v;
        }
        __syncwarp();
        int stf = fit_one<N>(ws, a, &itf);
        if (lane < kCoef) a.coef_f[cell * kCoef + lane] = ws.coef[lane];
        if (lane == 0) {
            a.status[cell * 2] = stv;
            a.status[cell * 2 + 1] = stf;
            atomicAdd(&a.counters[CNT_ITERS], (unsigned long long)(itv + itf));
            unsigned long long fb = (stv == 1) + (stf == 1);
            if (fb) atomicAdd(&a.counters[CNT_FALLBACK], fb);
            unsigned long long inv = (stv == 2) + (stf == 2);
            if (inv) atomicAdd(&a.counters[CNT_INVALID], inv);
        }
        __syncwarp();
    }
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

// index-space parameters of one Maxwellian for the exchange: the exponent
// at cell (i, j, k) is lognorm - 1/2 d^T Pt d with d = (i, j, k) - ic (ic =
// index of the peak); computed from the fit coefficients (eta, u0, sigma):
// q(w) = eta0 + lambda.w + w^T mu w has its peak at w* = -mu^-1 lambda / 2
// with value eta0 + lambda.w*/2, and w = w0 + h * index with h = dv/sigma.
struct MaxwIdx {
    double ic[3];
    double Pt[6];  // xx xy xz yy yz zz
    double lognorm;
    int valid;
};

__device__ void maxwellian_index_params(const double* k, int valid, const double* vmin, const double* dv,
                                        MaxwIdx* o) {
    o->valid = valid;
    if (!valid) return;
    double mu[9] = {k[4], 0.5 * k[5], 0.5 * k[6], 0.5 * k[5], k[7], 0.5 * k[8], 0.5 * k[6], 0.5 * k[8], k[9]};
    double mi[9];
    inv3(mu, mi);
    const double lam[3] = {k[1], k[2], k[3]};
    double ws[3], q = k[0];
    for (int a = 0; a < 3; ++a) {
        ws[a] = -0.5 * (mi[a * 3] * lam[0] + mi[a * 3 + 1] * lam[1] + mi[a * 3 + 2] * lam[2]);
        q += 0.5 * lam[a] * ws[a];
    }
    const double* u0 = k + 10;
    const double* sg = k + 13;
    double h[3];
    for (int a = 0; a < 3; ++a) {
        h[a] = dv[a] / sg[a];
        double w0 = (vmin[a] + 0.5 * dv[a] - u0[a]) / sg[a];
        o->ic[a] = (ws[a] - w0) / h[a];
    }
    o->Pt[0] = -2.0 * h[0] * h[0] * mu[0];
    o->Pt[1] = -2.0 * h[0] * h[1] * mu[1];
    o->Pt[2] = -2.0 * h[0] * h[2] * mu[2];
    o->Pt[3] = -2.0 * h[1] * h[1] * mu[4];
    o->Pt[4] = -2.0 * h[1] * h[2] * mu[5];
    o->Pt[5] = -2.0 * h[2] * h[2] * mu[8];
    o->lognorm = q;
}

// Maxwellian along the x line (j, k): values M_i for i = 0..N-1 by recurrence.
template <typename T, int N>
__device__ __forceinline__ void maxwellian_line(const MaxwIdx& p, int j, int k, T (&out)[N]) {
    if (!p.valid) {
#pragma unroll
        for (int i = 0; i < N; ++i) out[i] = T(0);
        return;
    }
    const T dy = (T)(j - p.ic[1]), dz = (T)(k - p.ic[2]);
    const T dx0 = (T)(0 - p.ic[0]);
    const T Pxx = (T)p.Pt[0], Pxy = (T)p.Pt[1], Pxz = (T)p.Pt[2];
    const T Pyy = (T)p.Pt[3], Pyz = (T)p.Pt[4], Pzz = (T)p.Pt[5];
    const T b = Pxy * dy + Pxz * dz;
    // exponent at i: -1/2 (Pxx dx^2 + 2 dx b + Pyy dy^2 + 2 Pyz dy dz + Pzz dz^2)
    const T q0 = T(-0.5) * (Pxx * dx0 * dx0 + T(2) * dx0 * b + Pyy * dy * dy + T(2) * Pyz * dy * dz + Pzz * dz * dz);
    T M = exp(q0 + (T)p.lognorm);
    T r = exp(T(-0.5) * Pxx * (T(2) * dx0 + T(1)) - b);
    const T rho = exp(-Pxx);
#pragma unroll
    for (int i = 0; i < N; ++i) {
        out[i] = M;
        M *= r;
        r *= rho;
    }
}

template <typename T, int N>
__global__ void exchange_kernel(ExchangeArgs a) {
    __shared__ MaxwIdx mp[2];
    __shared__ double red[20 * 32 + 20];
    __shared__ double ssum[32];
    __shared__ int sneg[32];
    T* f = reinterpret_cast<T*>(a.f);
    constexpr long long V = (long long)N * N * N;
    const int t = threadIdx.x;
    const int lane = t & 31, warp = t >> 5, nwarp = blockDim.x >> 5;
    const double vol = a.dv[0] * a.dv[1] * a.dv[2];
    for (long long cell = blockIdx.x; cell < a.ncell; cell += gridDim.x) {
        const int stv = a.status[cell * 2], stf = a.status[cell * 2 + 1];
        const bool skip = (stv == 2 || stf == 2);
        if (t < 2) maxwellian_index_params((t == 0 ? a.coef_v : a.coef_f) + cell * kCoef, (t == 0 ? stv : stf) != 2, a.vmin, a.dv, &mp[t]);
        __syncthreads();
        T r[N];
        const int j = t % N, k = t / N;
        const bool active = t < N * N;
        T lsum = T(0);
        int neg = 0;
        if (active) {
            const T* src = f + cell * V + (long long)(k * N + j) * N;
#pragma unroll
            for (int i = 0; i < N; ++i) r[i] = src[i];
            if (!skip) {
                T mv[N], mf[N];
                maxwellian_line<T, N>(mp[0], j, k, mv);
                maxwellian_line<T, N>(mp[1], j, k, mf);
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    r[i] = r[i] - mv[i] + mf[i];
                    neg |= r[i] < T(0);
                    lsum += fmax(r[i], T(0));
                }
            }
        }
        // block reduction: any negative, sum of the clipped values
        double s = warp_sum((double)lsum);
        int nn = __any_sync(0xffffffffu, neg);
        if (lane == 0) {
            ssum[warp] = s;
            sneg[warp] = nn;
        }
        __syncthreads();
        double tot = 0.0;
        int anyneg = 0;
        for (int w = 0; w < nwarp; ++w) {
            tot += ssum[w];
            anyneg |= sneg[w];
        }
        T scale = T(1);
        if (anyneg && !skip) {
            const double nV = a.vmom[cell * 20];
            scale = (T)(tot > 0.0 ? nV / (tot * vol) : 0.0);
            if (t == 0) atomicAdd(&a.counters[CNT_CLIPPED], 1ull);
        }
        T m[20];
#pragma unroll
        for (int q = 0; q < 20; ++q) m[q] = T(0);
        if (active) {
            T* dst = f + cell * V + (long long)(k * N + j) * N;
            const T c = T(0.5) * T(N - 1);
            T S0 = 0, S1 = 0, S2 = 0, S3 = 0;
#pragma unroll
            for (int i = 0; i < N; ++i) {
                T v = anyneg ? fmax(r[i], T(0)) * scale : r[i];
                dst[i] = v;
                T xi = T(i) - c;
                T v1 = v * xi, v2 = v1 * xi;
                S0 += v;
                S1 += v1;
                S2 += v2;
                S3 += v2 * xi;
            }
            if (a.mom_out) {
                const T e = T(j) - c, z = T(k) - c;
                const T e2 = e * e, z2 = z * z, ez = e * z;
                m[0] = S0; m[1] = S1; m[2] = e * S0; m[3] = z * S0;
                m[4] = S2; m[5] = e * S1; m[6] = z * S1; m[7] = e2 * S0; m[8] = ez * S0; m[9] = z2 * S0;
                m[10] = S3; m[11] = e * S2; m[12] = z * S2; m[13] = e2 * S1; m[14] = ez * S1; m[15] = z2 * S1;
                m[16] = e2 * e * S0; m[17] = e2 * z * S0; m[18] = e * z2 * S0; m[19] = z2 * z * S0;
            }
        }
        if (a.mom_out) {
#pragma unroll
            for (int q = 0; q < 20; ++q) {
                T v = m[q];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                m[q] = v;
            }
            if (lane == 0)
#pragma unroll
                for (int q = 0; q < 20; ++q) red[warp * 20 + q] = (double)m[q];
            __syncthreads();
            double* im = red + 20 * 32;
            if (t < 20) {
                double acc = 0.0;
                for (int w = 0; w < nwarp; ++w) acc += red[w * 20 + t];
                im[t] = acc;
            }
            __syncwarp();
            if (t < 20) {
                double acc = 0.0;
                for (int q = 0; q < a.conv.nterm[t]; ++q) acc += a.conv.coef[t][q] * im[a.conv.idx[t][q]];
                a.mom_out[cell * 20 + t] = acc;
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------- 1D1V

// One thread per cell: 3-parameter fits (n, u, Theta) by Newton in FP64 on
// the natural parameters of exp(e0 + e1 w + e2 w^2), then the exchange.
__device__ int fit1d(const double* target, const FitArgs& a, double* theta, int* iters) {
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
        for (int q = 0; q < 3; ++q) D[q] = 0.0;
        for (int q = 0; q < 5; ++q) G4[q] = 0.0;
        for (int i = 0; i < a.nv; ++i) {
            double w = w0 + i * h;
            double M = exp(e[0] + e[1] * w + e[2] * w * w) * a.dv[0];
            double p = M;
            for (int q = 0; q < 5; ++q) {
                if (q < 3) D[q] += p;
                G4[q] += p;
                p *= w;
            }
        }
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
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= a.ncell) return;
    double tv[3] = {a.vmom[c * 4], a.vmom[c * 4 + 1], a.vmom[c * 4 + 2]};
    const double nF = a.fluid[c * 3];
    const double scale = nF > 0.0 ? tv[0] / nF : 0.0;
    double tf[3];
    for (int q = 0; q < 3; ++q) tf[q] = a.fluid[c * 3 + q] * scale;
    double th[3];
    int itv, itf;
    int stv = fit1d(tv, a, th, &itv);
    for (int q = 0; q < 3; ++q) a.coef_v[c * kCoef + q] = th[q];
    int stf = fit1d(tf, a, th, &itf);
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

template <typename T>
__global__ void exchange1d_kernel(ExchangeArgs a) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= a.ncell) return;
    T* f = reinterpret_cast<T*>(a.f) + c * a.nv;
    const int stv = a.status[c * 2], stf = a.status[c * 2 + 1];
    if (stv != 2 && stf != 2) {
        const double* tv = a.coef_v + c * kCoef;
        const double* tf = a.coef_f + c * kCoef;
        bool neg = false;
        double sum = 0.0;
        for (int i = 0; i < a.nv; ++i) {
            double v = a.vmin[0] + (i + 0.5) * a.dv[0];
            double mv = tv[0] / sqrt(2.0 * M_PI * tv[2]) * exp(-0.5 * (v - tv[1]) * (v - tv[1]) / tv[2]);
            double mf = tf[0] / sqrt(2.0 * M_PI * tf[2]) * exp(-0.5 * (v - tf[1]) * (v - tf[1]) / tf[2]);
            T x = (T)((double)f[i] - mv + mf);
            f[i] = x;
            neg |= x < T(0);
            sum += x > T(0) ? (double)x : 0.0;
        }
        if (neg) {
            double sc = sum > 0.0 ? a.vmom[c * 4] / (sum * a.dv[0]) : 0.0;
            for (int i = 0; i < a.nv; ++i) f[i] = (T)(f[i] > T(0) ? (double)f[i] * sc : 0.0);
            atomicAdd(&a.counters[CNT_CLIPPED], 1ull);
        }
    }
    if (a.mom_out) {
        double m[4] = {0, 0, 0, 0};
        for (int q = 0; q < a.nv; ++q) {
            double v = a.vmin[0] + (q + 0.5) * a.dv[0], x = (double)f[q];
            m[0] += x; m[1] += v * x; m[2] += v * v * x; m[3] += v * v * v * x;
        }
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

template <int N>
static cudaError_t launch_fit_n(const FitArgs& a, cudaStream_t st) {
    const int threads = 128;  // 4 cells per CTA, one warp each
    long long blocks = (a.ncell + 3) / 4;
    long long cap = (long long)sm_count() * 16;
    if (blocks > cap) blocks = cap;
    fit_kernel<N><<<(unsigned)blocks, threads, 0, st>>>(a);
    count_launch();
    return cudaGetLastError();
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
        unsigned grid = (unsigned)((a.ncell + 127) / 128);
        fit1d_kernel<<<grid, 128, 0, st>>>(a);
        count_launch();
        return cudaGetLastError();
    }
    switch (a.nv) {
        case 8: return launch_fit_n<8>(a, st);
        case 12: return launch_fit_n<12>(a, st);
        case 16: return launch_fit_n<16>(a, st);
        case 20: return launch_fit_n<20>(a, st);
        case 24: return launch_fit_n<24>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int N>
static cudaError_t launch_exchange_n(const ExchangeArgs& a, cudaStream_t st) {
    const int threads = ((N * N + 31) / 32) * 32;
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
        unsigned grid = (unsigned)((a.ncell + 127) / 128);
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
