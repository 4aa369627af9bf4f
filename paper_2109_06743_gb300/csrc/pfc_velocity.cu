// Velocity-space PFC advection under the Lorentz force (paper Sec. 2.1) and
// the midpoint moments of f (Sec. 2.1), fused.
//
// Each spatial cell's velocity block (N^3 values) is staged in shared memory
// once; all velocity sweeps run there, so the pass moves f through HBM once
// (read + write). The velocity map of one time step is affine, V = R (v + h)
// + h (the Boris map, R a rotation about B, h = (q/m) E dt / 2). The paper
// splits it into 1D sweeps ("backsubstitution", not detailed in the paper);
// here R is factored exactly into five single-axis shears (rows p, b, c, b,
// p, with p the axis of the largest |B| component), each of which is a 1D
// PFC advection with a displacement that is constant along its line. The
// factors are computed per cell in FP64 by a small kernel, then the block
// kernel applies them with zero-flux boundaries at the velocity box.
//
// Shared-memory layout of a block: element (i, j, k) (i = v_x index fastest)
// at (k N + j)(N + 1) + i: x lines are padded to N+1 so that a warp walking
// 32 different lines hits distinct banks (32 consecutive v_z lines at fixed
// v_z index span 33 words: one bank is hit twice).
//
// FP32 blocks run velocity_pair_kernel (two lines per thread, packed FP32x2
// arithmetic, every line walked upwards); FP64 blocks run velocity_kernel
// (one line per thread, walked in the direction of its displacement).
#include "common.cuh"
#include "kernels.cuh"
#include "block_moments.cuh"
#include "f32x2.cuh"

namespace vl {

// --------------------------------------------------------------- shear factors

__device__ void cross3(const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// out[k][4] = (axis, coefficient of the lower other axis, of the higher one,
// constant): sweep k moves v_axis by c1 v_lo + c2 v_hi + c0.
__device__ void velocity_shears(double qm, double dt, const double* E, const double* B, int nshear,
                                double* out) {
    if (nshear == 3) {
        double w = qm * dt;
        double tab[3][4] = {{0, w * B[2], -w * B[1], w * E[0]},
                            {1, -w * B[2], w * B[0], w * E[1]},
                            {2, w * B[1], -w * B[0], w * E[2]}};
        for (int k = 0; k < 3; ++k)
            for (int q = 0; q < 4; ++q) out[k * 4 + q] = tab[k][q];
        return;
    }
    double t[3], s[3], tt = 0.0;
    for (int a = 0; a < 3; ++a) {
        t[a] = 0.5 * qm * dt * B[a];
        tt += t[a] * t[a];
    }
    for (int a = 0; a < 3; ++a) s[a] = 2.0 * t[a] / (1.0 + tt);
    // D = R - I, column by column: (e + e x t) x s
    double D[3][3];
    for (int col = 0; col < 3; ++col) {
        double e[3] = {0.0, 0.0, 0.0}, et[3], w[3], r[3];
        e[col] = 1.0;
        cross3(e, t, et);
        for (int a = 0; a < 3; ++a) w[a] = e[a] + et[a];
        cross3(w, s, r);
        for (int a = 0; a < 3; ++a) D[a][col] = r[a];
    }
    double h[3], bt[3];
    for (int a = 0; a < 3; ++a) h[a] = 0.5 * qm * dt * E[a];
    for (int a = 0; a < 3; ++a) bt[a] = D[a][0] * h[0] + D[a][1] * h[1] + D[a][2] * h[2] + 2.0 * h[a];
    // pivot axis: largest |B| component (first on ties)
    int p = 0;
    if (fabs(B[1]) > fabs(B[p])) p = 1;
    if (fabs(B[2]) > fabs(B[p])) p = 2;
    int perm[3] = {p, p == 0 ? 1 : 0, p == 2 ? 1 : 2};
    double M[3][3], dd0, dd1;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[i][j] = D[perm[i]][perm[j]] + (i == j ? 1.0 : 0.0);
    dd0 = D[perm[0]][perm[0]];
    dd1 = D[perm[1]][perm[1]];
    // op 1, row 0: least-norm combination of rows 1, 2 making M00 = 1
    double a1 = 0.0, b1 = 0.0;
    {
        double den = M[1][0] * M[1][0] + M[2][0] * M[2][0];
        if (den > 0.0) {
            a1 = -dd0 * M[1][0] / den;
            b1 = -dd0 * M[2][0] / den;
        }
        for (int col = 0; col < 3; ++col) M[0][col] += a1 * M[1][col] + b1 * M[2][col];
        M[0][0] = 1.0;
    }
    // op 2, row 1: rows 0, 2 making M10 = 0, M11 = 1
    double c2, d2;
    {
        double det = M[2][1] - M[2][0] * M[0][1];
        double r0 = -M[1][0], r1 = -dd1;
        if (det != 0.0) {
            d2 = (r1 - M[0][1] * r0) / det;
            c2 = r0 - d2 * M[2][0];
        } else {
            d2 = 0.0;
            c2 = r0;
        }
        for (int col = 0; col < 3; ++col) M[1][col] += c2 * M[0][col] + d2 * M[2][col];
        M[1][0] = 0.0;
        M[1][1] = 1.0;
    }
    // op 3, row 2: rows 0, 1 clearing M20, M21
    double e3 = -M[2][0];
    double g3 = -M[2][1] - e3 * M[0][1];
    for (int col = 0; col < 3; ++col) M[2][col] += e3 * M[0][col] + g3 * M[1][col];
    // op 4, row 1: row 2 clearing M12
    double c4 = -M[1][2];
    for (int col = 0; col < 3; ++col) M[1][col] += c4 * M[2][col];
    // op 5, row 0: rows 1, 2 clearing M01, M02
    double a5 = -M[0][1], b5 = -M[0][2];

    // sweeps in application order (inverse operations 5, 4, 3, 2, 1); per
    // sweep: permuted row and coefficients on the permuted columns
    double lin[5][3] = {{0.0, -a5, -b5}, {0.0, 0.0, -c4}, {-e3, -g3, 0.0}, {-c2, 0.0, -d2}, {0.0, -a1, -b1}};
    int prow[5] = {0, 1, 2, 1, 0};
    // constants (sweeps 2, 3, 4) reproduce the translation bt
    double bp[3] = {bt[perm[0]], bt[perm[1]], bt[perm[2]]};
    double k2 = bp[2];
    double k3 = bp[1] + d2 * k2;
    double k4 = bp[0] - (a1 * d2 - b1) * k2 + a1 * k3;
    double cst[5] = {0.0, 0.0, k2, k3, k4};
    for (int k = 0; k < 5; ++k) {
        int r = prow[k];
        int o1 = r == 0 ? 1 : 0, o2 = r == 2 ? 1 : 2;  // other permuted indices, o1 < o2
        int ax = perm[r];
        double cl = lin[k][o1], ch = lin[k][o2];
        if (perm[o1] > perm[o2]) {  // order the coefficients by physical axis
            double tmp = cl;
            cl = ch;
            ch = tmp;
        }
        out[k * 4 + 0] = ax;
        out[k * 4 + 1] = cl;
        out[k * 4 + 2] = ch;
        out[k * 4 + 3] = cst[k];
    }
}

__global__ void shear_setup_kernel(const double* eb, double* shears, long long ncell, double qm, double dt,
                                   int nshear) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    velocity_shears(qm, dt, eb + c * 6, eb + c * 6 + 3, nshear, shears + c * 20);
}

// ------------------------------------------------------------- line update

template <typename T>
__device__ __forceinline__ T phi_lim(T alpha, T A, T B, T fm, T f0, T fp) {
    T up = fmin(fp - f0, T(2) * f0);
    T dn = fmax(f0 - fm, T(-2) * f0);
    return alpha * (f0 + A * up + B * dn);
}

template <int N>
__device__ __forceinline__ int padded(int i, int j, int k) {
    return (k * N + j) * (N + 1) + i;
}

// Apply one shear along velocity axis AX to the block in smem: every thread
// owns one line (lo, hi = indices of the lower and higher other axes) and
// runs the zero-flux PFC step on it in registers. The line is walked in the
// frame where the displacement is positive (a signed shared-memory stride);
// everything that would leave through the far boundary piles up in the last
// cell and cells the profile has left become zero. When no line of the warp
// moves by a whole cell (the usual case) the shifted write-back reduces to a
// plain one.
template <typename T, int N, int AX>
__device__ __forceinline__ void apply_shear_ax(T* blk, const T* sh, const T* vc, const T* inv_dv) {
    constexpr int ST = AX == 0 ? 1 : (AX == 1 ? N + 1 : N * (N + 1));
    const int t = threadIdx.x;
    const bool active = t < N * N;
    const int lo = active ? t % N : 0, hi = active ? t / N : 0;
    constexpr int alo = AX == 0 ? 1 : 0, ahi = AX == 2 ? 1 : 2;
    const int base = AX == 0 ? padded<N>(0, lo, hi) : (AX == 1 ? padded<N>(lo, 0, hi) : padded<N>(lo, hi, 0));
    const T vlo = vc[alo * N + lo], vhi = vc[ahi * N + hi];
    const T c = (sh[1] * vlo + sh[2] * vhi + sh[3]) * inv_dv[AX];
    const bool fwd = c >= T(0);
    T ca = fwd ? c : -c;
    // beyond N cells everything piles up in the last cell anyway; clamping in
    // floating point also maps NaN to N, so the int conversion is always safe
    if (!(ca < T(N))) ca = T(N);
    const int s = (int)floor(ca);
    const T alpha = ca - (T)s;
    const int sst = fwd ? ST : -ST;
    T* line = blk + (fwd ? base : base + (N - 1) * ST);
    const bool whole = __ballot_sync(0xffffffffu, active && s != 0) != 0u;
    if (!active) return;
    T r[N];
#pragma unroll
    for (int q = 0; q < N; ++q) r[q] = line[q * sst];
    const T A = (T(1) - alpha) * (T(2) - alpha) / T(6);
    const T B = (T(1) - alpha) * (T(1) + alpha) / T(6);
    T phi_prev = T(0), old_prev = T(0), phi = T(0);
#pragma unroll
    for (int q = 0; q < N; ++q) {
        const T fp = q + 1 < N ? r[q + 1] : T(0);
        phi = phi_lim<T>(alpha, A, B, old_prev, r[q], fp);
        const T g = r[q] - phi + phi_prev;
        phi_prev = phi;
        old_prev = r[q];
        r[q] = g;
    }
    if (!whole) {
#pragma unroll
        for (int q = 0; q < N - 1; ++q) line[q * sst] = r[q];
        line[(N - 1) * sst] = r[N - 1] + phi;
        return;
    }
    T acc = T(0);
    T* shifted = line + s * sst;
#pragma unroll
    for (int q = 0; q < N; ++q) {
        if (q + s < N - 1) shifted[q * sst] = r[q];
        else acc += r[q];
    }
    line[(N - 1) * sst] = acc + phi;
#pragma unroll
    for (int p = 0; p < N - 1; ++p)
        if (p < s) line[p * sst] = T(0);
}

// sh: (axis, c_lo, c_hi, c_0) in T; vc[3][N]: cell-centre velocities;
// inv_dv[3]: 1 / dv
template <typename T, int N>
__device__ __forceinline__ void apply_shear(T* blk, const T* sh, const T* vc, const T* inv_dv) {
    const int axis = (int)sh[0];
    if (axis == 0) apply_shear_ax<T, N, 0>(blk, sh, vc, inv_dv);
    else if (axis == 1) apply_shear_ax<T, N, 1>(blk, sh, vc, inv_dv);
    else apply_shear_ax<T, N, 2>(blk, sh, vc, inv_dv);
}

// ---------------------------------------------------------------- moments

// Raw moments of the block in smem (padded layout) reduced over the CTA
// (line sums along v_x, see block_moments.cuh).
template <typename T, int N>
__device__ void block_moments(const T* blk, double* red, double* out, const MomConv& conv) {
    const int t = threadIdx.x;
    T m[20];
#pragma unroll
    for (int a = 0; a < 20; ++a) m[a] = T(0);
    if (t < N * N) {
        const int j = t % N, k = t / N;
        const T c = T(0.5) * T(N - 1);
        T S0 = 0, S1 = 0, S2 = 0, S3 = 0;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            T v = blk[padded<N>(i, j, k)];
            T xi = T(i) - c;
            T v1 = v * xi, v2 = v1 * xi;
            S0 += v;
            S1 += v1;
            S2 += v2;
            S3 += v2 * xi;
        }
        line_products<T, N>(m, S0, S1, S2, S3, j, k);
    }
    reduce_moments<T>(m, red, out, conv);
}

void make_mom_conv(const double* vmin, const double* dv, int n, MomConv* out) {
    static const int P[20][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0}, {1, 1, 0}, {1, 0, 1},
                                 {0, 2, 0}, {0, 1, 1}, {0, 0, 2}, {3, 0, 0}, {2, 1, 0}, {2, 0, 1}, {1, 2, 0},
                                 {1, 1, 1}, {1, 0, 2}, {0, 3, 0}, {0, 2, 1}, {0, 1, 2}, {0, 0, 3}};
    static const double binom[4][4] = {{1, 0, 0, 0}, {1, 1, 0, 0}, {1, 2, 1, 0}, {1, 3, 3, 1}};
    double vc[3];
    for (int a = 0; a < 3; ++a) vc[a] = vmin[a] + 0.5 * n * dv[a];
    const double vol = dv[0] * dv[1] * dv[2];
    auto ipow = [](double x, int k) {
        double r = 1.0;
        for (int q = 0; q < k; ++q) r *= x;
        return r;
    };
    for (int o = 0; o < 20; ++o) {
        int nt = 0;
        for (int p = 0; p <= P[o][0]; ++p)
            for (int q = 0; q <= P[o][1]; ++q)
                for (int r = 0; r <= P[o][2]; ++r) {
                    double w = binom[P[o][0]][p] * ipow(vc[0], P[o][0] - p) * ipow(dv[0], p) *
                               binom[P[o][1]][q] * ipow(vc[1], P[o][1] - q) * ipow(dv[1], q) *
                               binom[P[o][2]][r] * ipow(vc[2], P[o][2] - r) * ipow(dv[2], r) * vol;
                    if (w == 0.0) continue;
                    int idx = 0;
                    for (int u = 0; u < 20; ++u)
                        if (P[u][0] == p && P[u][1] == q && P[u][2] == r) idx = u;
                    out->coef[o][nt] = w;
                    out->idx[o][nt] = (unsigned char)idx;
                    ++nt;
                }
        out->nterm[o] = (unsigned char)nt;
    }
}

// ---------------------------------------------------------------- kernels

constexpr int vel_threads(int n) { return ((n * n + 31) / 32) * 32; }

// Block copies with the CTA's compile-time thread count, so the loops unroll
// and (for N^2 a multiple of 32) every index step is a constant.
template <typename T, int N, int NTH = vel_threads(N)>
__device__ __forceinline__ void load_block(T* blk, const T* src) {
    constexpr int V = N * N * N;
#pragma unroll 4
    for (int e = threadIdx.x; e < V; e += NTH) {
        int i = e % N, jk = e / N;
        blk[jk * (N + 1) + i] = src[e];
    }
}

// asynchronous element copies of one block into the padded layout (the
// padding breaks 16-byte alignment of the rows, so element-sized copies)
template <typename T, int N, int NTH = vel_threads(N)>
__device__ __forceinline__ void prefetch_block(T* blk, const T* src) {
    constexpr int V = N * N * N;
#pragma unroll 4
    for (int e = threadIdx.x; e < V; e += NTH) {
        const int i = e % N, jk = e / N;
        const unsigned d = (unsigned)__cvta_generic_to_shared(blk + jk * (N + 1) + i);
        if (sizeof(T) == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src + e) : "memory");
        else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src + e) : "memory");
    }
}

// The same copies when the thread count is a multiple of the row length and
// the block a multiple of the thread count: every thread keeps one column of
// rows, so both addresses step by compile-time constants (no per-element
// index arithmetic).
template <int N, int NTH>
constexpr bool rows_tile() { return NTH % N == 0 && (N * N * N) % NTH == 0; }
template <int N, int NTH>
constexpr bool groups_tile() { return (4 * NTH) % N == 0 && (N * N * N / 4) % NTH == 0; }

template <int N, int NTH>
__device__ __forceinline__ void prefetch_block_rows(float* blk, const float* src) {
    constexpr int R = NTH / N, U = N * N * N / NTH;
    const int t = threadIdx.x;
    const unsigned d = (unsigned)__cvta_generic_to_shared(blk + (t / N) * (N + 1) + t % N);
    const float* g = src + t;
#pragma unroll
    for (int u = 0; u < U; ++u)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d + 4u * (unsigned)(u * R * (N + 1))),
                     "l"(g + u * NTH)
                     : "memory");
}

template <int N, int NTH>
__device__ __forceinline__ void store_block_groups(float* dst, const float* blk) {
    constexpr int U = N * N * N / 4 / NTH, R = 4 * NTH / N;
    const int t = threadIdx.x;
    const float* row = blk + (4 * t / N) * (N + 1) + (4 * t) % N;
    float* g = dst + 4 * t;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const float* q = row + u * R * (N + 1);
        *reinterpret_cast<float4*>(g + u * 4 * NTH) = make_float4(q[0], q[1], q[2], q[3]);
    }
}

// write the block back; with vec (16-byte aligned f) in 16-byte stores: a
// row holds N values (N a multiple of 4), so each group of 16 bytes comes
// from one padded row
template <typename T, int N, int NTH = vel_threads(N)>
__device__ __forceinline__ void store_block(T* dst, const T* blk, bool vec) {
    constexpr int V = N * N * N;
    constexpr int per = 16 / (int)sizeof(T);
    static_assert(N % 4 == 0, "rows of whole 16-byte groups");
    if (!vec) {
#pragma unroll 4
        for (int e = threadIdx.x; e < V; e += NTH) {
            const int i = e % N, jk = e / N;
            dst[e] = blk[jk * (N + 1) + i];
        }
        return;
    }
#pragma unroll 4
    for (int g = threadIdx.x; g < V / per; g += NTH) {
        const int e = g * per;
        const int i = e % N, jk = e / N;
        const T* row = blk + jk * (N + 1) + i;
        if (sizeof(T) == 4) {
            const float4 v = make_float4((float)row[0], (float)row[1], (float)row[2], (float)row[3]);
            *reinterpret_cast<float4*>(dst + e) = v;
        } else {
            const double2 v = make_double2((double)row[0], (double)row[1]);
            *reinterpret_cast<double2*>(dst + e) = v;
        }
    }
}

// One CTA per velocity block at a time (persistent over cells); the FP64
// pass. With a.nbuf == 2 the next cell's block is copied in while the
// current one is advected. Registers are capped at 128 per thread where the
// block size allows, so that several CTAs share an SM.
constexpr int vel_min_blocks(int n, int es) {
    return 65536 / ((es == 8 ? 128 : 64) * vel_threads(n)) > 0 ? 65536 / ((es == 8 ? 128 : 64) * vel_threads(n)) : 1;
}
template <typename T, int N>
__global__ void __launch_bounds__(vel_threads(N), vel_min_blocks(N, sizeof(T))) velocity_kernel(VelocityArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int BLK = N * N * (N + 1);
    T* const buf0 = reinterpret_cast<T*>(smem_raw);
    T* const buf1 = buf0 + BLK;
    double* red = reinterpret_cast<double*>(smem_raw + sizeof(T) * BLK * a.nbuf);
    T* sh = reinterpret_cast<T*>(red + 20 * 32 + 20);  // [20] shears of the cell
    T* vc = sh + 20;                                    // [3][N] cell-centre velocities
    T* inv_dv = vc + 3 * N;                             // [3]
    T* f = reinterpret_cast<T*>(a.f);
    constexpr long long V = (long long)N * N * N;
    const bool two = a.nbuf == 2;
    for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) {
        const int ax = q / N, i = q % N;
        vc[q] = (T)(a.vmin[ax] + (i + 0.5) * a.dv[ax]);
    }
    if (threadIdx.x < 3) inv_dv[threadIdx.x] = (T)(1.0 / a.dv[threadIdx.x]);
    long long cell = blockIdx.x;
    if (two && cell < a.ncell) prefetch_block<T, N>(buf0, f + cell * V);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    for (int it = 0; cell < a.ncell; cell += gridDim.x, ++it) {
        T* blk = (two && (it & 1)) ? buf1 : buf0;
        if (two) {
            const long long nx = cell + gridDim.x;
            if (nx < a.ncell) prefetch_block<T, N>((it & 1) ? buf0 : buf1, f + nx * V);
            asm volatile("cp.async.commit_group;\n" ::: "memory");
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            load_block<T, N>(blk, f + cell * V);
        }
        if (threadIdx.x < 20) sh[threadIdx.x] = (T)a.shears[cell * 20 + threadIdx.x];
        __syncthreads();
        for (int k = 0; k < a.nshear; ++k) {
            apply_shear<T, N>(blk, sh + 4 * k, vc, inv_dv);
            __syncthreads();
        }
        if (a.mom_out) block_moments<T, N>(blk, red, a.mom_out + cell * 20, a.conv);
        store_block<T, N>(f + cell * V, blk, a.vec != 0);
        __syncthreads();
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// ------------------------------------------------ FP32: two lines per thread
//
// The FP32 pass pairs the lines of every sweep two to a thread and updates
// both with packed FP32x2 arithmetic (add/sub/mul/fma.f32x2), which halves
// the issue slots of the line update; the limiter's min/max stay scalar.
//
// Every line is walked in increasing index order whatever the sign of its
// displacement, so that each shared-memory access is a compile-time offset
// from the line's start. With a_i = f_{i+1} - f_i (zero ghosts outside the
// box), U_i = min(a_i, 2 f_i) and D_i = max(a_{i-1}, -2 f_i), the flux that
// leaves cell i in the direction of the displacement is
//   c >= 0: alpha (f_i + A U_i + B D_i), out through face i + 1/2,
//   c <  0: alpha (f_i - A D_i - B U_i), out through face i - 1/2,
// (A = (1 - alpha)(2 - alpha)/6, B = (1 - alpha)(1 + alpha)/6; the second
// is the first one mirrored). With phi_i = a0 f_i + P U_i + Q D_i the flux
// through face i + 1/2 counted in the +v direction (a0, P, Q = alpha,
// alpha A, alpha B for c >= 0; -alpha, alpha B, alpha A for c < 0), the new
// value of cell q is f_q + c0 phi_q + cm phi_{q-1} + cp phi_{q+1}, with
// (c0, cm, cp) = (-1, 1, 0) or (1, 0, -1). At the box faces nothing flows
// out: the first cell drops its own term for c < 0 (coefficient -cm), the
// last one for c >= 0 (coefficient -cp).

namespace pair {

using x2::add;
using x2::fma;
using x2::mul;
using x2::neg;
using x2::sub;

constexpr int threads(int n) { return ((n * n / 2 + 31) / 32) * 32; }
constexpr int warps(int n) { return threads(n) / 32; }
// CTAs per SM the register cap is sized for
constexpr int min_blocks(int n) { return n <= 8 ? 16 : (n <= 12 ? 6 : (n <= 16 ? 5 : 2)); }

// physical exponents (x, y, z) of moment o, packed x + 4 y + 16 z
__host__ __device__ constexpr int mono_exp(int o) {
    constexpr int e[20] = {0, 1, 4, 16, 2, 5, 17, 8, 20, 32, 3, 6, 18, 9, 21, 33, 12, 24, 36, 48};
    return e[o];
}

// both lines' coefficients at once, in packed arithmetic: with sg = +-1 the
// sign of the displacement, h = (1 - alpha)/6 and t = sg (1/2 - alpha),
// alpha A and alpha B are alpha h (3/2 + t) and alpha h (3/2 - t) in the
// order (P, Q) of the formula above
struct PairCoef {
    float2 a0, P, Q, c0, cm, cp;
    int s1, s2;
    bool f1, f2;
};

template <int N>
__device__ __forceinline__ PairCoef pair_coef(float2 c) {
    PairCoef k;
    k.f1 = c.x >= 0.0f;
    k.f2 = c.y >= 0.0f;
    const float2 sg = make_float2(k.f1 ? 1.0f : -1.0f, k.f2 ? 1.0f : -1.0f);
    // clamped at N cells (fminf also maps NaN to N)
    const float2 ca = make_float2(fminf(fabsf(c.x), float(N)), fminf(fabsf(c.y), float(N)));
    const float2 fl = make_float2(floorf(ca.x), floorf(ca.y));
    k.s1 = (int)fl.x;
    k.s2 = (int)fl.y;
    const float2 al = sub(ca, fl);
    const float2 sixth = make_float2(1.0f / 6.0f, 1.0f / 6.0f), half = make_float2(0.5f, 0.5f);
    const float2 h = fma(neg(al), sixth, sixth);
    const float2 t = mul(sg, sub(half, al));
    const float2 ah = mul(al, h);
    const float2 th = make_float2(1.5f, 1.5f);
    k.P = mul(ah, add(th, t));
    k.Q = mul(ah, sub(th, t));
    k.a0 = mul(sg, al);
    k.c0 = neg(sg);
    k.cm = fma(sg, half, half);
    k.cp = sub(k.cm, make_float2(1.0f, 1.0f));
    return k;
}

// integer part of the displacement of one line: g (the fractional update,
// both box faces closed) moves s cells in the direction of the displacement,
// what would leave the box piles up in the last cell, the cells it leaves
// become zero (the one-dimensional sweep at any displacement, Sec. 2.1)
template <int N, int ST, int C>
__device__ __forceinline__ void shift_store(float* line, const float2 (&g)[N], int s, bool fwd) {
    auto at = [&](int q) -> float { return C == 0 ? g[q].x : g[q].y; };
    if (s == 0) {
#pragma unroll
        for (int q = 0; q < N; ++q) line[q * ST] = at(q);
        return;
    }
    float acc = 0.0f;
    if (fwd) {
#pragma unroll
        for (int q = 0; q < N; ++q) {
            if (q + s < N - 1) line[(q + s) * ST] = at(q);
            else acc += at(q);
        }
        line[(N - 1) * ST] = acc;
#pragma unroll
        for (int p = 0; p < N - 1; ++p)
            if (p < s) line[p * ST] = 0.0f;
    } else {
#pragma unroll
        for (int q = N - 1; q >= 0; --q) {
            if (q - s > 0) line[(q - s) * ST] = at(q);
            else acc += at(q);
        }
        line[0] = acc;
#pragma unroll
        for (int p = 1; p < N; ++p)
            if (p > N - 1 - s) line[p * ST] = 0.0f;
    }
}

// the 20 raw-moment products of one line along axis AX with centred sums
// S[0..3] at centred indices e (lower other axis), z (higher other axis)
template <int AX>
__device__ __forceinline__ void line_moments(float (&m)[20], const float (&S)[4], float e, float z) {
    constexpr int alo = AX == 0 ? 1 : 0, ahi = AX == 2 ? 1 : 2;
    const float pe[4] = {1.0f, e, e * e, e * e * e};
    const float pz[4] = {1.0f, z, z * z, z * z * z};
#pragma unroll
    for (int o = 0; o < 20; ++o) {
        const int x = mono_exp(o);
        const int ex[3] = {x & 3, (x >> 2) & 3, (x >> 4) & 3};
        const int a = ex[AX], b = ex[alo], c = ex[ahi];
        if (b == 0 && c == 0) m[o] += S[a];
        else if (c == 0) m[o] = fmaf(S[a], pe[b], m[o]);
        else if (b == 0) m[o] = fmaf(S[a], pz[c], m[o]);
        else m[o] = fmaf(S[a], pe[b] * pz[c], m[o]);
    }
}

// One sweep along velocity axis AX over the pair of lines (lo1, hi1),
// (lo2, hi2) of this thread. RAGGED: some threads hold fewer than two lines
// (v1, v2 false), their loads give zero and their stores are skipped. MOM:
// this is the block's last sweep: the 20 moment products of the result are
// formed from the registers and reduced over the CTA into out.
template <int N, int AX, bool RAGGED, bool MOM>
__device__ __forceinline__ void sweep(float* blk, const float* sh, const float* vc, const float* inv_dv, int lo1,
                                      int hi1, int lo2, int hi2, bool v1, bool v2, float (&m)[20]) {
    constexpr int ST = AX == 0 ? 1 : (AX == 1 ? N + 1 : N * (N + 1));
    constexpr int alo = AX == 0 ? 1 : 0, ahi = AX == 2 ? 1 : 2;
    auto start = [](int lo, int hi) {
        return AX == 0 ? padded<N>(0, lo, hi) : (AX == 1 ? padded<N>(lo, 0, hi) : padded<N>(lo, hi, 0));
    };
    float* const L1 = blk + start(lo1, hi1);
    float* const L2 = blk + start(lo2, hi2);
    const float idv = inv_dv[AX];
    const PairCoef k = pair_coef<N>(make_float2((sh[1] * vc[alo * N + lo1] + sh[2] * vc[ahi * N + hi1] + sh[3]) * idv,
                                                (sh[1] * vc[alo * N + lo2] + sh[2] * vc[ahi * N + hi2] + sh[3]) * idv));
    const float2 a0 = k.a0, P = k.P, Q = k.Q, c0 = k.c0, cm = k.cm, cp = k.cp;
    const bool whole = __ballot_sync(0xffffffffu, (v1 && k.s1 != 0) || (v2 && k.s2 != 0)) != 0u;
    float2 r[N];
#pragma unroll
    for (int q = 0; q < N; ++q) {
        r[q].x = (!RAGGED || v1) ? L1[q * ST] : 0.0f;
        r[q].y = (!RAGGED || v2) ? L2[q * ST] : 0.0f;
    }
    float2 a_prev = r[0];  // a_{-1} = f_0 - 0
    float2 ph1 = make_float2(0.0f, 0.0f), ph2 = ph1;  // phi_{q-1}, phi_{q-2}
#pragma unroll
    for (int q = 0; q < N; ++q) {
        const float2 f = r[q];
        const float2 a = q + 1 < N ? sub(r[q + 1], f) : neg(f);
        const float2 f2 = add(f, f);
        const float2 U = make_float2(fminf(a.x, f2.x), fminf(a.y, f2.y));
        const float2 D = make_float2(fmaxf(a_prev.x, -f2.x), fmaxf(a_prev.y, -f2.y));
        const float2 ph = fma(Q, D, fma(P, U, mul(a0, f)));
        if (q == 1) r[0] = fma(cp, ph, fma(neg(cm), ph1, r[0]));
        else if (q >= 2) r[q - 1] = fma(cp, ph, fma(cm, ph2, fma(c0, ph1, r[q - 1])));
        ph2 = ph1;
        ph1 = ph;
        a_prev = a;
    }
    r[N - 1] = fma(cm, ph2, fma(neg(cp), ph1, r[N - 1]));
    if (!whole) {
#pragma unroll
        for (int q = 0; q < N; ++q) {
            if (!RAGGED || v1) L1[q * ST] = r[q].x;
            if (!RAGGED || v2) L2[q * ST] = r[q].y;
        }
    } else {
        if (!RAGGED || v1) shift_store<N, ST, 0>(L1, r, k.s1, k.f1);
        if (!RAGGED || v2) shift_store<N, ST, 1>(L2, r, k.s2, k.f2);
        if (MOM) {
            // the thread's own stores: read back the shifted lines
#pragma unroll
            for (int q = 0; q < N; ++q) {
                r[q].x = (!RAGGED || v1) ? L1[q * ST] : 0.0f;
                r[q].y = (!RAGGED || v2) ? L2[q * ST] : 0.0f;
            }
        }
    }
    if (MOM) {
        // centred sums S_p = sum_q xi_q^p f_q, xi_q = q - (N-1)/2, folded over
        // the mirror pairs q, N-1-q (xi_{N-1-q} = -xi_q)
        float2 s0 = make_float2(0.0f, 0.0f);
        float S1x = 0.0f, S1y = 0.0f, S2x = 0.0f, S2y = 0.0f, S3x = 0.0f, S3y = 0.0f;
#pragma unroll
        for (int q = 0; q < N / 2; ++q) {
            const float xi = (float)q - 0.5f * (float)(N - 1);
            const float2 u = add(r[q], r[N - 1 - q]);
            const float2 d = sub(r[q], r[N - 1 - q]);
            s0 = add(s0, u);
            S1x = fmaf(d.x, xi, S1x);
            S1y = fmaf(d.y, xi, S1y);
            S2x = fmaf(u.x, xi * xi, S2x);
            S2y = fmaf(u.y, xi * xi, S2y);
            S3x = fmaf(d.x, xi * xi * xi, S3x);
            S3y = fmaf(d.y, xi * xi * xi, S3y);
        }
        const float cc = 0.5f * (float)(N - 1);
        const float Sa[4] = {s0.x, S1x, S2x, S3x}, Sb[4] = {s0.y, S1y, S2y, S3y};
        line_moments<AX>(m, Sa, (float)lo1 - cc, (float)hi1 - cc);
        line_moments<AX>(m, Sb, (float)lo2 - cc, (float)hi2 - cc);
    }
}

template <int N, bool RAGGED, bool MOM>
__device__ __forceinline__ void sweep_axis(int axis, float* blk, const float* sh, const float* vc,
                                           const float* inv_dv, int lo1, int hi1, int lo2, int hi2, bool v1, bool v2,
                                           float (&m)[20]) {
    if (axis == 0) sweep<N, 0, RAGGED, MOM>(blk, sh, vc, inv_dv, lo1, hi1, lo2, hi2, v1, v2, m);
    else if (axis == 1) sweep<N, 1, RAGGED, MOM>(blk, sh, vc, inv_dv, lo1, hi1, lo2, hi2, v1, v2, m);
    else sweep<N, 2, RAGGED, MOM>(blk, sh, vc, inv_dv, lo1, hi1, lo2, hi2, v1, v2, m);
}

}  // namespace pair

// One CTA per velocity block at a time (persistent over cells), as
// velocity_kernel, with the FP32 two-lines-per-thread sweeps. Thread t of
// warp w holds lines w 64 + lane and w 64 + 32 + lane (line = hi N + lo), so
// each shared-memory instruction of a warp touches 32 consecutive lines.
template <int N>
__global__ void __launch_bounds__(pair::threads(N), pair::min_blocks(N)) velocity_pair_kernel(VelocityArgs a) {
    constexpr int NTH = pair::threads(N);
    constexpr bool RAGGED = (N * N) % 64 != 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int BLK = N * N * (N + 1);
    float* const buf0 = reinterpret_cast<float*>(smem_raw);
    float* const buf1 = buf0 + BLK;
    double* red = reinterpret_cast<double*>(smem_raw + sizeof(float) * BLK * a.nbuf);
    float* sh = reinterpret_cast<float*>(red + 20 * pair::warps(N) + 20);  // [20] shears of the cell
    float* vc = sh + 20;                                                   // [3][N] cell-centre velocities
    float* inv_dv = vc + 3 * N;                                            // [3]
    float* f = reinterpret_cast<float*>(a.f);
    constexpr long long V = (long long)N * N * N;
    const bool two = a.nbuf == 2;
    for (int q = threadIdx.x; q < 3 * N; q += NTH) {
        const int ax = q / N, i = q % N;
        vc[q] = (float)(a.vmin[ax] + (i + 0.5) * a.dv[ax]);
    }
    if (threadIdx.x < 3) inv_dv[threadIdx.x] = (float)(1.0 / a.dv[threadIdx.x]);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m1 = warp * 64 + lane, m2 = m1 + 32;
    const bool v1 = m1 < N * N, v2 = m2 < N * N;
    const int lo1 = v1 ? m1 % N : 0, hi1 = v1 ? m1 / N : 0;
    const int lo2 = v2 ? m2 % N : 0, hi2 = v2 ? m2 / N : 0;
    long long cell = blockIdx.x;
    auto prefetch = [](float* blk, const float* src) {
        if constexpr (rows_tile<N, NTH>()) prefetch_block_rows<N, NTH>(blk, src);
        else prefetch_block<float, N, NTH>(blk, src);
    };
    if (two && cell < a.ncell) prefetch(buf0, f + cell * V);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    for (int it = 0; cell < a.ncell; cell += gridDim.x, ++it) {
        float* blk = (two && (it & 1)) ? buf1 : buf0;
        if (two) {
            const long long nx = cell + gridDim.x;
            if (nx < a.ncell) prefetch((it & 1) ? buf0 : buf1, f + nx * V);
            asm volatile("cp.async.commit_group;\n" ::: "memory");
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            load_block<float, N, NTH>(blk, f + cell * V);
        }
        if (threadIdx.x < 20) sh[threadIdx.x] = (float)a.shears[cell * 20 + threadIdx.x];
        __syncthreads();
        double* out = a.mom_out ? a.mom_out + cell * 20 : nullptr;
        for (int k = 0; k < a.nshear; ++k) {
            const float* s = sh + 4 * k;
            const int axis = (int)s[0];
            float m[20];
#pragma unroll
            for (int o = 0; o < 20; ++o) m[o] = 0.0f;
            if (out && k == a.nshear - 1) {
                pair::sweep_axis<N, RAGGED, true>(axis, blk, s, vc, inv_dv, lo1, hi1, lo2, hi2, v1, v2, m);
                reduce_moments<float, pair::warps(N)>(m, red, out, a.conv);
            } else {
                pair::sweep_axis<N, RAGGED, false>(axis, blk, s, vc, inv_dv, lo1, hi1, lo2, hi2, v1, v2, m);
            }
            __syncthreads();
        }
        if (groups_tile<N, NTH>() && a.vec) store_block_groups<N, NTH>(f + cell * V, blk);
        else store_block<float, N, NTH>(f + cell * V, blk, a.vec != 0);
        __syncthreads();
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <typename T, int N>
__global__ void moments_kernel(MomentArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* blk = reinterpret_cast<T*>(smem_raw);
    double* red = reinterpret_cast<double*>(smem_raw + sizeof(T) * N * N * (N + 1));
    const T* f = reinterpret_cast<const T*>(a.f);
    constexpr long long V = (long long)N * N * N;
    for (long long cell = blockIdx.x; cell < a.ncell; cell += gridDim.x) {
        load_block<T, N>(blk, f + cell * V);
        __syncthreads();
        block_moments<T, N>(blk, red, a.mom_out + cell * 20, a.conv);
        __syncthreads();
    }
}

// ------------------------------------------------------------------- 1D1V

// One thread per spatial cell: zero-flux PFC step of the velocity line with
// c = (q/m) E dt / dv, straight from global memory (1D1V lines are short).
template <typename T>
__global__ void velocity1d_kernel(VelocityArgs a) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= a.ncell) return;
    T* f = reinterpret_cast<T*>(a.f) + c * a.nv;
    const int n = a.nv;
    double cc = a.qm * a.eb[c * 6] * a.dt / a.dv[0];
    bool fwd = cc >= 0.0;
    double ca = fwd ? cc : -cc;
    if (!(ca < (double)n)) ca = (double)n;
    int s = (int)floor(ca);
    T alpha = (T)(ca - s);
    const T A = (T(1) - alpha) * (T(2) - alpha) / T(6);
    const T B = (T(1) - alpha) * (T(1) + alpha) / T(6);
    T g[64];
    auto at = [&](int q) -> T { return (q < 0 || q >= n) ? T(0) : f[fwd ? q : n - 1 - q]; };
    T phi_prev = T(0), phi = T(0);
    for (int q = 0; q < n; ++q) {
        phi = phi_lim<T>(alpha, A, B, at(q - 1), at(q), at(q + 1));
        g[q] = at(q) - phi + phi_prev;
        phi_prev = phi;
    }
    T acc = T(0);
    for (int p = 0; p < n; ++p) {
        int q = p - s;
        T v = (q >= 0) ? g[q] : T(0);
        if (p == n - 1) {
            for (int qq = (q >= 0 ? q : 0); qq < n; ++qq) acc += g[qq];
            v = acc + phi;
        }
        f[fwd ? p : n - 1 - p] = v;
    }
    if (a.mom_out) {
        double m[4] = {0, 0, 0, 0};
        for (int q = 0; q < n; ++q) {
            double v = a.vmin[0] + (q + 0.5) * a.dv[0], x = (double)f[q];
            m[0] += x; m[1] += v * x; m[2] += v * v * x; m[3] += v * v * v * x;
        }
        for (int p = 0; p < 4; ++p) a.mom_out[c * 4 + p] = m[p] * a.dv[0];
    }
}

template <typename T>
__global__ void moments1d_kernel(MomentArgs a) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= a.ncell) return;
    const T* f = reinterpret_cast<const T*>(a.f) + c * a.nv;
    double m[4] = {0, 0, 0, 0};
    for (int q = 0; q < a.nv; ++q) {
        double v = a.vmin[0] + (q + 0.5) * a.dv[0], x = (double)f[q];
        m[0] += x; m[1] += v * x; m[2] += v * v * x; m[3] += v * v * v * x;
    }
    for (int p = 0; p < 4; ++p) a.mom_out[c * 4 + p] = m[p] * a.dv[0];
}

// ---------------------------------------------------------------- launchers

static int g_num_sms = 0;
static int num_sms() {
    if (g_num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 148;
    }
    return g_num_sms;
}

template <typename T, int N>
static cudaError_t launch_velocity_n(const VelocityArgs& a, cudaStream_t st) {
    const int threads = ((N * N + 31) / 32) * 32;
    const size_t blk = sizeof(T) * N * N * (N + 1);
    VelocityArgs b = a;
    // double buffering while two buffers leave room for two CTAs per SM
    b.nbuf = 2 * blk <= 100 * 1024 ? 2 : 1;
    b.vec = reinterpret_cast<uintptr_t>(a.f) % 16 == 0;
    size_t smem = blk * b.nbuf + sizeof(double) * (20 * 32 + 20) + sizeof(T) * (20 + 3 * N + 3);
    cudaFuncSetAttribute(velocity_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, velocity_kernel<T, N>, threads, smem);
    if (per_sm < 1) per_sm = 1;
    long long grid = (long long)num_sms() * per_sm;
    if (grid > a.ncell) grid = a.ncell;
    velocity_kernel<T, N><<<(unsigned)grid, threads, smem, st>>>(b);
    count_launch();
    return cudaGetLastError();
}

template <int N>
static cudaError_t launch_velocity_pair(const VelocityArgs& a, cudaStream_t st) {
    const int threads = pair::threads(N);
    const size_t blk = sizeof(float) * N * N * (N + 1);
    VelocityArgs b = a;
    b.nbuf = 2 * blk <= 100 * 1024 ? 2 : 1;
    b.vec = reinterpret_cast<uintptr_t>(a.f) % 16 == 0;
    size_t smem = blk * b.nbuf + sizeof(double) * (20 * pair::warps(N) + 20) + sizeof(float) * (20 + 3 * N + 3);
    cudaFuncSetAttribute(velocity_pair_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, velocity_pair_kernel<N>, threads, smem);
    if (per_sm < 1) per_sm = 1;
    long long grid = (long long)num_sms() * per_sm;
    if (grid > a.ncell) grid = a.ncell;
    velocity_pair_kernel<N><<<(unsigned)grid, threads, smem, st>>>(b);
    count_launch();
    return cudaGetLastError();
}

template <typename T, int N>
static cudaError_t launch_moments_n(const MomentArgs& a, cudaStream_t st) {
    const int threads = ((N * N + 31) / 32) * 32;
    size_t smem = sizeof(T) * N * N * (N + 1) + sizeof(double) * (20 * 32 + 20);
    cudaFuncSetAttribute(moments_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, moments_kernel<T, N>, threads, smem);
    if (per_sm < 1) per_sm = 1;
    long long grid = (long long)num_sms() * per_sm;
    if (grid > a.ncell) grid = a.ncell;
    moments_kernel<T, N><<<(unsigned)grid, threads, smem, st>>>(a);
    count_launch();
    return cudaGetLastError();
}

#define VL_DISPATCH_N(FN, T, nv, ...)                \
    switch (nv) {                                    \
        case 8: return FN<T, 8>(__VA_ARGS__);        \
        case 12: return FN<T, 12>(__VA_ARGS__);      \
        case 16: return FN<T, 16>(__VA_ARGS__);      \
        case 20: return FN<T, 20>(__VA_ARGS__);      \
        case 24: return FN<T, 24>(__VA_ARGS__);      \
        default: return cudaErrorInvalidValue;       \
    }

cudaError_t launch_velocity(const VelocityArgs& a, int nvdim, int precision, cudaStream_t st) {
    if (nvdim == 1) {
        int threads = 128;
        unsigned grid = (unsigned)((a.ncell + threads - 1) / threads);
        if (precision == 64) velocity1d_kernel<double><<<grid, threads, 0, st>>>(a);
        else velocity1d_kernel<float><<<grid, threads, 0, st>>>(a);
        count_launch();
        return cudaGetLastError();
    }
    {
        int threads = 128;
        unsigned grid = (unsigned)((a.ncell + threads - 1) / threads);
        shear_setup_kernel<<<grid, threads, 0, st>>>(a.eb, a.shears, a.ncell, a.qm, a.dt, a.nshear);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (precision == 64) { VL_DISPATCH_N(launch_velocity_n, double, a.nv, a, st); }
    switch (a.nv) {
        case 8: return launch_velocity_pair<8>(a, st);
        case 12: return launch_velocity_pair<12>(a, st);
        case 16: return launch_velocity_pair<16>(a, st);
        case 20: return launch_velocity_pair<20>(a, st);
        case 24: return launch_velocity_pair<24>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_moments(const MomentArgs& a, int nvdim, int precision, cudaStream_t st) {
    if (nvdim == 1) {
        int threads = 128;
        unsigned grid = (unsigned)((a.ncell + threads - 1) / threads);
        if (precision == 64) moments1d_kernel<double><<<grid, threads, 0, st>>>(a);
        else moments1d_kernel<float><<<grid, threads, 0, st>>>(a);
        count_launch();
        return cudaGetLastError();
    }
    if (precision == 64) { VL_DISPATCH_N(launch_moments_n, double, a.nv, a, st); }
    VL_DISPATCH_N(launch_moments_n, float, a.nv, a, st);
}

}  // namespace vl
