// Spatial PFC sweeps (paper Sec. 2.1: PFC scheme of Filbet, Sonnendruecker
// and Bertrand 2001; Sec. 3.3: reflecting walls in y).
//
// A tile is one spatial line (a y row for the x sweep, an x column for the y
// sweep) times W velocity columns: rows along the sweep axis, each row made
// of contiguous 128-byte runs of the velocity block (with reflecting walls:
// two adjacent v_y rows and their two mirror rows). Persistent CTAs walk the tiles; each tile is staged in
// shared memory with 16-byte cp.async copies, double buffered, so the copy of
// tile t+1 is in flight while tile t is computed. Each thread walks a segment
// of one column with a sliding window and writes the result straight back to
// global memory; a CTA reads its whole tile before writing it, so the sweep
// is in place.
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

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory"); }

// velocity index of tile column col, and the column holding its v_y mirror
__device__ __forceinline__ bool col_vi(const SpaceSweepArgs& a, int chunk, int col, int* vi, int* mcol) {
    if (a.mode == 0) {
        const int v = chunk * a.ncol + col;
        *vi = v;
        *mcol = col;
        return v < a.V;
    }
    if (a.mode == 2) {
        // reflecting walls: rows j, j + 1 of the lower v_y half and their
        // mirrors jm - 1, jm (jm = nvy - 1 - j), two contiguous runs of 2 nvx
        const int nvx = a.nvx, pairs = a.nvy / 4;
        const int k = chunk / pairs, j = 2 * (chunk % pairs), jm = a.nvy - 1 - j;
        if (col < 2 * nvx) {
            const int r = col / nvx;
            *vi = (k * a.nvy + j) * nvx + col;
            *mcol = (3 - r) * nvx + col % nvx;
        } else {
            const int c2 = col - 2 * nvx, r = c2 / nvx;
            *vi = (k * a.nvy + jm - 1) * nvx + c2;
            *mcol = (1 - r) * nvx + c2 % nvx;
        }
        return true;
    }
    const int half = (a.nvy + 1) / 2;
    const int k = chunk / half, j = chunk % half;
    const int jm = a.nvy - 1 - j;
    if (col < a.nvx) {
        *vi = (k * a.nvy + j) * a.nvx + col;
        *mcol = (jm == j) ? col : col + a.nvx;
        return true;
    }
    if (jm == j || col >= 2 * a.nvx) return false;
    *vi = (k * a.nvy + jm) * a.nvx + (col - a.nvx);
    *mcol = col - a.nvx;
    return true;
}

// issue the copies of one tile: 16-byte cp.async chunks when every column
// run starts on a 16-byte boundary and spans a multiple of 16 bytes (a.vec),
// else plain element loads
template <typename T>
__device__ __forceinline__ void load_tile(const SpaceSweepArgs& a, const T* f, T* tile, int tidx) {
    const int chunk = tidx % a.nchunks;
    const long long base = (long long)(tidx / a.nchunks) * a.line_stride;
    int vi;
    int mc;
    if (a.vec) {
        constexpr int per = 16 / sizeof(T);
        const int cpr = a.ncol / per;  // chunks per row
        for (int idx = threadIdx.x; idx < a.n * cpr; idx += blockDim.x) {
            const int r = idx / cpr, c = (idx - r * cpr) * per;
            if (col_vi(a, chunk, c, &vi, &mc))
                cp_async16(tile + r * a.ncol + c, f + base + (long long)r * a.row_stride + vi);
        }
    } else {
        for (int idx = threadIdx.x; idx < a.n * a.ncol; idx += blockDim.x) {
            const int r = idx / a.ncol, c = idx - r * a.ncol;
            if (col_vi(a, chunk, c, &vi, &mc)) tile[idx] = f[base + (long long)r * a.row_stride + vi];
        }
    }
}

// Per-column constants of the update, one entry per velocity index along the
// sweep axis (computed once per CTA in FP64, used in T)
template <typename T>
struct ColumnStep {
    T alpha, A, B;
    int s, fwd;
};

template <typename T>
__global__ void __launch_bounds__(1024) pfc_space_kernel(SpaceSweepArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* f = reinterpret_cast<T*>(a.f);
    const int ncol = a.ncol, n = a.n;
    T* const buf0 = reinterpret_cast<T*>(smem_raw);
    T* const buf1 = buf0 + (size_t)n * ncol;
    ColumnStep<T>* steps = reinterpret_cast<ColumnStep<T>*>(smem_raw + (size_t)a.nbuf * n * ncol * sizeof(T));
    for (int ia = threadIdx.x; ia < a.axis_mod; ia += blockDim.x) {
        // displacement of velocity index ia in cells
        const double c = (a.vmin_a + (ia + 0.5) * a.dv_a) * a.dt_over_h;
        const bool fwd = c >= 0.0;
        double ca = fwd ? c : -c;
        // periodic lines: a shift by whole line lengths is the identity;
        // walls: the host guarantees ca + 3 <= n. Clamp before the int
        // conversion.
        if (!a.wall) ca = fmod(ca, (double)n);
        if (!(ca <= (double)n)) ca = (double)n;
        const int s = (int)floor(ca);
        const T alpha = (T)(ca - s);
        ColumnStep<T> cs;
        cs.alpha = alpha;
        cs.A = (T(1) - alpha) * (T(2) - alpha) / T(6);
        cs.B = (T(1) - alpha) * (T(1) + alpha) / T(6);
        cs.s = s;
        cs.fwd = fwd;
        steps[ia] = cs;
    }
    const int ntiles = a.nchunks * a.nlines;  // < 2^31, checked on the host
    const int nseg = blockDim.x / ncol;
    const int col = threadIdx.x % ncol;
    const int seg = threadIdx.x / ncol;
    const int L = (n + nseg - 1) / nseg;

    const bool two = a.nbuf == 2;
    int t = blockIdx.x;
    if (two && t < ntiles) load_tile<T>(a, f, buf0, t);
    cp_async_commit();
    for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
        if (two) {
            const int tn = t + gridDim.x;
            if (tn < ntiles) load_tile<T>(a, f, (it & 1) ? buf0 : buf1, tn);
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            load_tile<T>(a, f, buf0, t);
            cp_async_commit();
            cp_async_wait<0>();
        }
        __syncthreads();
        const T* tile = (two && (it & 1)) ? buf1 : buf0;
        const int chunk = t % a.nchunks;
        const long long base = (long long)(t / a.nchunks) * a.line_stride;
        int vi;
        int mcol;
        if (seg < nseg && col_vi(a, chunk, col, &vi, &mcol)) {
            const ColumnStep<T> cs = steps[(vi / a.axis_div) % a.axis_mod];
            const bool fwd = cs.fwd != 0;
            const int s = cs.s;
            const T alpha = cs.alpha, A = cs.A, B = cs.B;
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
            const int k0 = seg * L;
            const int k1 = min(n, k0 + L);
            if (k0 < k1) {
                int j = k0 - s;
                T fm1 = fetch(j - 1), f0 = fetch(j), fp1 = fetch(j + 1);
                T phim = pfc_phi<T>(alpha, A, B, fetch(j - 2), fm1, f0);
                // output walks the line in the frame's direction
                T* out = f + base + vi + (long long)(fwd ? k0 : n - 1 - k0) * a.row_stride;
                const long long os = fwd ? a.row_stride : -a.row_stride;
                // at step k the window needs the value at frame index k - s + 2:
                // inside the line for s - 2 <= k <= n - 3 + s, where it is read
                // straight from the tile with a signed stride; the few steps
                // outside take the periodic or mirrored value
                const int ka = max(k0, min(k1, s - 2));
                const int kb = max(ka, min(k1, n - 2 + s));
                auto advance = [&](T next) {
                    const T phi = pfc_phi<T>(alpha, A, B, fm1, f0, fp1);
                    *out = f0 - phi + phim;
                    out += os;
                    fm1 = f0;
                    f0 = fp1;
                    fp1 = next;
                    phim = phi;
                };
                int k = k0;
                for (; k < ka; ++k) advance(fetch(k - s + 2));
                {
                    const int ts = fwd ? ncol : -ncol;
                    const T* src = tile + (fwd ? col : (n - 1) * ncol + col) + (k - s + 2) * ts;
#pragma unroll 4
                    for (; k < kb; ++k) {
                        const T next = *src;
                        src += ts;
                        advance(next);
                    }
                }
                for (; k < k1; ++k) advance(fetch(k - s + 2));
            }
        }
        __syncthreads();  // the buffer of tile t is refilled in a later iteration
    }
    cp_async_wait<0>();
}

static int g_sms = 0;

cudaError_t launch_pfc_space(const SpaceSweepArgs& a, int precision, cudaStream_t st) {
    if (g_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_sms <= 0) g_sms = 148;
    }
    const size_t es = precision == 64 ? sizeof(double) : sizeof(float);
    const size_t smem = (size_t)a.nbuf * a.n * a.ncol * es + (size_t)a.axis_mod * (es == 8 ? sizeof(ColumnStep<double>) : sizeof(ColumnStep<float>));
    const long long ntiles = (long long)a.nchunks * a.nlines;
    // one thread per (column, segment of about 16 cells), up to 1024 threads:
    // short segments give each SM enough independent sliding windows to hide
    // the shared-memory latency of the window updates
    int nseg = (a.n + 15) / 16;
    if (nseg > 1024 / a.ncol) nseg = 1024 / a.ncol;
    if (nseg < 1) nseg = 1;
    const int threads = a.ncol * nseg;
    int per_sm = 0;
    if (precision == 64) {
        cudaFuncSetAttribute(pfc_space_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pfc_space_kernel<double>, threads, smem);
    } else {
        cudaFuncSetAttribute(pfc_space_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pfc_space_kernel<float>, threads, smem);
    }
    if (per_sm < 1) per_sm = 1;
    long long grid = (long long)g_sms * per_sm;
    if (grid > ntiles) grid = ntiles;
    if (precision == 64) pfc_space_kernel<double><<<(unsigned)grid, threads, smem, st>>>(a);
    else pfc_space_kernel<float><<<(unsigned)grid, threads, smem, st>>>(a);
    count_launch();
    return cudaGetLastError();
}

}  // namespace vl
