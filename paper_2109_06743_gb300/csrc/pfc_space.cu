// Spatial PFC sweeps (paper Sec. 2.1: PFC scheme of Filbet, Sonnendruecker
// and Bertrand 2001; Sec. 3.3: reflecting walls in y).
//
// One CTA owns one spatial line (a y row for the x sweep, an x column for the
// y sweep) for a tile of velocity columns. The whole line of the tile is
// staged in shared memory (rows along the sweep axis, columns = velocity
// indices, so every global access is a contiguous run of the velocity block),
// then each thread walks a segment of one column with a sliding window and
// writes the result straight back to global memory. Since a CTA reads
// everything it writes before writing, the sweep is in place.
//
// For a displacement c = v dt / dx = s + alpha (alpha in [0,1)) the PFC update
// is f_i <- g_{i-s}, g_j = f_j - phi_j + phi_{j-1}, with the limited flux
//   phi_j = alpha (f_j + A min(f_{j+1}-f_j, 2 f_j) + B max(f_j-f_{j-1}, -2 f_j)),
//   A = (1-alpha)(2-alpha)/6, B = (1-alpha)(1+alpha)/6,
// which is the positivity-limited form of Filbet et al. written without
// divisions (eps+ (f_{j+1}-f_j) = min(f_{j+1}-f_j, 2 f_j), and likewise for
// eps-). A negative displacement is the same update on the reversed line.
#include "common.cuh"
#include "kernels.cuh"

namespace vl {

template <typename T>
__device__ __forceinline__ T pfc_phi(T alpha, T A, T B, T fm, T f0, T fp) {
    T up = fmin(fp - f0, T(2) * f0);
    T dn = fmax(f0 - fm, T(-2) * f0);
    return alpha * (f0 + A * up + B * dn);
}

template <typename T>
__global__ void __launch_bounds__(256) pfc_space_kernel(SpaceSweepArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* tile = reinterpret_cast<T*>(smem_raw);
    T* f = reinterpret_cast<T*>(a.f);
    const int ncol = a.ncol;
    const int n = a.n;
    const long long base = (long long)blockIdx.y * a.line_stride;
    const int chunk = blockIdx.x;

    // column -> velocity index (and its v_y mirror within the tile)
    auto col_vi = [&](int col, long long* vi, int* mcol) -> bool {
        if (a.mode == 0) {
            long long v = (long long)chunk * ncol + col;
            *vi = v;
            *mcol = col;
            return v < a.V;
        }
        int half = (a.nvy + 1) / 2;
        int k = chunk / half, j = chunk % half;
        int jm = a.nvy - 1 - j;
        if (col < a.nvx) {
            *vi = ((long long)k * a.nvy + j) * a.nvx + col;
            *mcol = (jm == j) ? col : col + a.nvx;
            return true;
        }
        if (jm == j || col >= 2 * a.nvx) return false;
        *vi = ((long long)k * a.nvy + jm) * a.nvx + (col - a.nvx);
        *mcol = col - a.nvx;
        return true;
    };

    // stage the tile: rows along the line, contiguous velocity columns
    for (int idx = threadIdx.x; idx < n * ncol; idx += blockDim.x) {
        int r = idx / ncol, col = idx - r * ncol;
        long long vi;
        int mc;
        if (col_vi(col, &vi, &mc)) tile[idx] = f[base + (long long)r * a.row_stride + vi];
    }
    __syncthreads();

    const int nseg = blockDim.x / ncol;
    const int col = threadIdx.x % ncol;
    const int seg = threadIdx.x / ncol;
    if (seg >= nseg) return;
    long long vi;
    int mcol;
    if (!col_vi(col, &vi, &mcol)) return;

    // displacement of this column in cells
    int ia = (int)((vi / a.axis_div) % a.axis_mod);
    double c = (a.vmin_a + (ia + 0.5) * a.dv_a) * a.dt_over_h;
    const bool fwd = c >= 0.0;
    double ca = fwd ? c : -c;
    // periodic lines: a shift by whole line lengths is the identity; walls:
    // the host guarantees ca + 3 <= n. Clamp before the int conversion.
    if (!a.wall) ca = fmod(ca, (double)n);
    if (!(ca <= (double)n)) ca = (double)n;
    const int s = (int)floor(ca);
    const T alpha = (T)(ca - s);
    const T A = (T(1) - alpha) * (T(2) - alpha) / T(6);
    const T B = (T(1) - alpha) * (T(1) + alpha) / T(6);

    // value at reversed-frame index j (physical p = j forward, n-1-j reversed)
    auto fetch = [&](int j) -> T {
        int p = fwd ? j : n - 1 - j;
        if (p >= 0 && p < n) return tile[p * ncol + col];
        if (!a.wall) {
            p %= n;
            if (p < 0) p += n;
            return tile[p * ncol + col];
        }
        p = p < 0 ? -1 - p : 2 * n - 1 - p;  // mirror row, v_y -> -v_y column
        return tile[p * ncol + mcol];
    };

    const int L = (n + nseg - 1) / nseg;
    const int k0 = seg * L;
    const int k1 = min(n, k0 + L);
    if (k0 >= k1) return;
    int j = k0 - s;
    T fm2 = fetch(j - 2), fm1 = fetch(j - 1), f0 = fetch(j), fp1 = fetch(j + 1);
    T phim = pfc_phi<T>(alpha, A, B, fm2, fm1, f0);
    for (int k = k0; k < k1; ++k) {
        T phi = pfc_phi<T>(alpha, A, B, fm1, f0, fp1);
        T g = f0 - phi + phim;
        int i = fwd ? k : n - 1 - k;
        f[base + (long long)i * a.row_stride + vi] = g;
        ++j;
        fm2 = fm1;
        fm1 = f0;
        f0 = fp1;
        fp1 = fetch(j + 1);
        phim = phi;
    }
}

cudaError_t launch_pfc_space(const SpaceSweepArgs& a, int precision, cudaStream_t st) {
    size_t es = precision == 64 ? sizeof(double) : sizeof(float);
    size_t smem = (size_t)a.n * a.ncol * es;
    dim3 grid(a.nchunks, a.nlines);
    if (precision == 64) {
        cudaFuncSetAttribute(pfc_space_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        pfc_space_kernel<double><<<grid, 256, smem, st>>>(a);
    } else {
        cudaFuncSetAttribute(pfc_space_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        pfc_space_kernel<float><<<grid, 256, smem, st>>>(a);
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace vl
