// Fused spatial PFC sweeps: x then y in one pass (paper Sec. 2.1, the
// directional splitting of the Vlasov step; Sec. 3.3, reflecting walls in y).
//
// The result equals pfc_advect_x along x followed by pfc_advect_x along y,
// element for element and with the same arithmetic, but f crosses HBM once
// (read f_in, write f_out) instead of twice. Because neighbouring tiles read
// each other's cells as halos, the pass is out of place.
//
// A CTA owns a spatial tile of TX x TY cells times ncol contiguous velocity
// columns (128 bytes per cell). Phase X: for every row the y sweep will look
// at (the TY tile rows plus hy = s_y,max + 2 halo rows on each side; beyond a
// wall, the mirror row in the v_y-mirrored column) the x-advected values at
// the tile's TX columns are computed straight from global memory (periodic
// wrap in x) and kept in shared memory. Phase Y: every (x, column) line of
// that buffer is advected along y and written to f_out.
//
// Each job (a segment of SEG outputs of one line) reads its SEG + 3 inputs in
// the frame of its displacement: with c = s + alpha, output k of the frame
// needs inputs k - s - 2 .. k - s + 1, so input q of the job is frame cell
// q - s - 2 and every index below is a compile-time constant; a negative
// displacement walks the line backwards.
//
// Two kernels: pfc_space_xy_tma_kernel (persistent; the input box of a tile,
// halos included, is one TMA tensor copy into shared memory, issued two tiles
// ahead into a double buffer and completed on an mbarrier; only the cells a
// tensor copy cannot express -- periodic images in x and y, mirror rows at a
// wall -- are patched in with plain loads) for x and y shifts up to 2 cells;
// pfc_space_xy_kernel (one CTA per tile, inputs read straight from global
// memory) for any shift.
#include <cuda.h>

#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace vl {

namespace {

template <typename T>
__device__ __forceinline__ T phi_xy(T alpha, T A, T B, T fm, T f0, T fp) {
    T up = fmin(fp - f0, T(2) * f0);
    T dn = fmax(f0 - fm, T(-2) * f0);
    return alpha * (f0 + A * up + B * dn);
}

template <typename T>
struct AxisStep {
    T alpha, A, B;
    int s, fwd;
};

// displacement constants of one velocity index along an axis, as the
// single-axis sweep computes them (FP64, reduced modulo the line length on
// periodic lines)
template <typename T>
__device__ AxisStep<T> axis_step(double vmin, double dv, double dt_over_h, int i, int n, bool wall) {
    const double c = (vmin + (i + 0.5) * dv) * dt_over_h;
    const bool fwd = c >= 0.0;
    double ca = fwd ? c : -c;
    if (!wall) ca = fmod(ca, (double)n);
    if (!(ca <= (double)n)) ca = (double)n;
    const int s = (int)floor(ca);
    const T alpha = (T)(ca - s);
    AxisStep<T> r;
    r.alpha = alpha;
    r.A = (T(1) - alpha) * (T(2) - alpha) / T(6);
    r.B = (T(1) - alpha) * (T(1) + alpha) / T(6);
    r.s = s;
    r.fwd = fwd;
    return r;
}

// SEG outputs of one line from in[0 .. SEG + 2] (frame order)
template <typename T, int SEG>
__device__ __forceinline__ void pfc_segment(const AxisStep<T>& st, const T (&in)[SEG + 3], T (&out)[SEG]) {
    T phim = phi_xy<T>(st.alpha, st.A, st.B, in[0], in[1], in[2]);
#pragma unroll
    for (int k = 0; k < SEG; ++k) {
        const T phi = phi_xy<T>(st.alpha, st.A, st.B, in[k + 1], in[k + 2], in[k + 3]);
        out[k] = in[k + 2] - phi + phim;
        phim = phi;
    }
}

// The same update in physical order, for both directions at once. With
// U_j = min(f_{j+1} - f_j, 2 f_j) and D_j = max(f_j - f_{j-1}, -2 f_j) (both
// independent of the direction), the limited flux of cell j is
// Phi_j = alpha (f_j + P U_j + Q D_j) with (P, Q) = (A, B) for a positive
// displacement and (-B, -A) for a negative one (reversing the line swaps the
// neighbours, which maps U to -D and D to -U exactly). A window w[0 .. SEG+3]
// starting at physical cell i0 - s - 2 (positive) or i0 + s - 2 (negative)
// gives the outputs at i0 .. i0 + SEG - 1 as
//   out_k = w_{k+2} - Phi_{k+2} + Phi_{k+1}   (positive: inflow from the left)
//   out_k = w_{k+2} - Phi_{k+2} + Phi_{k+3}   (negative: inflow from the right)
// so loads and stores use compile-time offsets in both cases.
template <typename T>
struct ColStep {
    T alpha, P, Q;
    int off;  // window start relative to the first output cell: -s-2 or s-2
    int fwd;
};

template <typename T>
__device__ ColStep<T> col_step(const AxisStep<T>& a) {
    ColStep<T> r;
    r.alpha = a.alpha;
    r.P = a.fwd ? a.A : -a.B;
    r.Q = a.fwd ? a.B : -a.A;
    r.off = a.fwd ? -a.s - 2 : a.s - 2;
    r.fwd = a.fwd;
    return r;
}

template <typename T, int SEG>
__device__ __forceinline__ void pfc_window(const ColStep<T>& st, const T (&w)[SEG + 4], T (&out)[SEG]) {
    T phi[SEG + 3];
#pragma unroll
    for (int j = 1; j <= SEG + 2; ++j) {
        const T two = T(2) * w[j];
        const T U = fmin(w[j + 1] - w[j], two);
        const T D = fmax(w[j] - w[j - 1], -two);
        phi[j] = st.alpha * (w[j] + st.P * U + st.Q * D);
    }
#pragma unroll
    for (int k = 0; k < SEG; ++k) out[k] = w[k + 2] - phi[k + 2] + (st.fwd ? phi[k + 1] : phi[k + 3]);
}

__device__ __forceinline__ int wrap(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// Phase Y of a tile: every (x, column) line of xs ([ty + 2 hy][tx][ncol],
// x-advected) is advected along y and its ty cells are written to f_out.
template <typename T, int SEG>
__device__ __forceinline__ void phase_y(const SpaceXYArgs& a, const T* xs, const AxisStep<T>* sty, int chunk, int x0,
                                        int y0, T* __restrict__ fout) {
    const int ncol = a.ncol, tx = a.tx, hy = a.hy;
    const long long V = a.V;
    const int nsy = a.ty / SEG;
    const int jobs_y = tx * nsy * ncol;
    for (int job = threadIdx.x; job < jobs_y; job += blockDim.x) {
        const int c = job % ncol;
        const int rest = job / ncol;
        const int xx = rest % tx, seg = rest / tx;
        const long long vi = (long long)chunk * ncol + c;
        if (vi >= V) continue;
        const AxisStep<T> st = sty[(vi / a.nvx) % a.nvy];
        const int ys0 = seg * SEG;
        // xs row of input q: fwd hy + ys0 - s - 2 + q, backward hy + ys0 + SEG + 1 + s - q
        const int dir = st.fwd ? 1 : -1;
        const int r0 = st.fwd ? hy + ys0 - st.s - 2 : hy + ys0 + SEG + 1 + st.s;
        const T* src = xs + ((size_t)r0 * tx + xx) * ncol + c;
        const int sstep = dir * tx * ncol;
        T in[SEG + 3];
#pragma unroll
        for (int q = 0; q < SEG + 3; ++q) in[q] = src[q * sstep];
        T out[SEG];
        pfc_segment<T, SEG>(st, in, out);
        const int yfirst = y0 + (st.fwd ? ys0 : ys0 + SEG - 1);
        T* o = fout + ((long long)yfirst * a.nx + x0 + xx) * V + vi;
        const long long ostep = (long long)dir * a.nx * V;
#pragma unroll
        for (int k = 0; k < SEG; ++k) o[k * ostep] = out[k];
    }
}

// source of the value the y sweep sees at row gy (possibly outside the
// domain) in velocity column vi: the row itself, its periodic image, or
// beyond a wall the mirror row in the v_y-mirrored column
__device__ __forceinline__ void row_source(const SpaceXYArgs& a, int gy, long long vi, int* sy, long long* svi) {
    *sy = gy;
    *svi = vi;
    if (gy >= 0 && gy < a.ny) return;
    if (a.wall) {
        // the velocity box is symmetric in v_y
        *sy = gy < 0 ? -1 - gy : 2 * a.ny - 1 - gy;
        const long long ix = vi % a.nvx, iy = (vi / a.nvx) % a.nvy, iz = vi / ((long long)a.nvx * a.nvy);
        *svi = (iz * a.nvy + (a.nvy - 1 - iy)) * a.nvx + ix;
    } else {
        *sy = wrap(gy, a.ny);
    }
}

}  // namespace

template <typename T, int SEG>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 2 : 1) pfc_space_xy_kernel(SpaceXYArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int ncol = a.ncol, tx = a.tx, ty = a.ty, hy = a.hy;
    const int rows = ty + 2 * hy;
    T* const xs = reinterpret_cast<T*>(smem_raw);  // [rows][tx][ncol]
    AxisStep<T>* const stx = reinterpret_cast<AxisStep<T>*>(smem_raw + sizeof(T) * (size_t)rows * tx * ncol);
    AxisStep<T>* const sty = stx + a.nvx;
    for (int i = threadIdx.x; i < a.nvx + a.nvy; i += blockDim.x) {
        if (i < a.nvx) stx[i] = axis_step<T>(a.vminx, a.dvx, a.cx, i, a.nx, false);
        else sty[i - a.nvx] = axis_step<T>(a.vminy, a.dvy, a.cy, i - a.nvx, a.ny, a.wall != 0);
    }
    __syncthreads();

    const int ntx = a.nx / tx, nty = a.ny / ty;
    const long long tile = blockIdx.x;
    const int tix = (int)(tile % ntx);
    const int tiy = (int)((tile / ntx) % nty);
    const int chunk = (int)(tile / ((long long)ntx * nty));
    const int x0 = tix * tx, y0 = tiy * ty;
    const long long V = a.V;
    const T* __restrict__ fin = reinterpret_cast<const T*>(a.f_in);
    T* __restrict__ fout = reinterpret_cast<T*>(a.f_out);

    // ---- phase X: x-advected rows y0 - hy .. y0 + ty + hy - 1 into xs
    const int nsx = tx / SEG;
    const int jobs_x = rows * nsx * ncol;
    for (int job = threadIdx.x; job < jobs_x; job += blockDim.x) {
        const int c = job % ncol;
        const int rest = job / ncol;
        const int seg = rest % nsx, r = rest / nsx;
        const long long vi = (long long)chunk * ncol + c;
        if (vi >= V) continue;
        int sy;
        long long svi;
        row_source(a, y0 - hy + r, vi, &sy, &svi);
        const AxisStep<T> st = stx[vi % a.nvx];
        const int xs0 = seg * SEG;
        // x of input q: fwd x0 + xs0 - s - 2 + q, backward x0 + xs0 + SEG + 1 + s - q
        const int dir = st.fwd ? 1 : -1;
        const int g0 = st.fwd ? x0 + xs0 - st.s - 2 : x0 + xs0 + SEG + 1 + st.s;
        const int glast = g0 + dir * (SEG + 2);
        const T* row = fin + (long long)sy * a.nx * V + svi;
        T in[SEG + 3];
        if (min(g0, glast) >= 0 && max(g0, glast) < a.nx) {
            const T* p = row + (long long)g0 * V;
            const long long step = dir * V;
#pragma unroll
            for (int q = 0; q < SEG + 3; ++q) in[q] = __ldg(p + q * step);
        } else {
#pragma unroll
            for (int q = 0; q < SEG + 3; ++q) in[q] = __ldg(row + (long long)wrap(g0 + dir * q, a.nx) * V);
        }
        T out[SEG];
        pfc_segment<T, SEG>(st, in, out);
        T* dst = xs + ((size_t)r * tx + (st.fwd ? xs0 : xs0 + SEG - 1)) * ncol + c;
        const int dstep = dir * ncol;
#pragma unroll
        for (int k = 0; k < SEG; ++k) dst[k * dstep] = out[k];
    }
    __syncthreads();

    // ---- phase Y: advect every (x, column) line of xs along y, write f_out
    phase_y<T, SEG>(a, xs, sty, chunk, x0, y0, fout);
}

// ---------------------------------------------------------------- TMA path

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(tc::smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// box of the tensor map at (c0, c1, c2) (innermost first) into shared memory
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(tc::smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(tc::smem_addr(bar))
        : "memory");
}

// polls of an mbarrier before a tile copy counts as lost (far beyond any
// real copy time; each poll is a bounded hardware wait)
constexpr uint32_t kCopyWaitPolls = 1u << 20;

#ifndef VL_XY_TX
#define VL_XY_TX 16
#endif
#ifndef VL_XY_TY
#define VL_XY_TY 16
#endif
#ifndef VL_XY_NT
#define VL_XY_NT 1024
#endif

// Shared memory: [2 mbarriers | pad to 128][S0][S1][xs][x steps][y steps];
// S = the input box [TY + 2 hy][TX + 2 hx][NCOL] of one tile. The tile
// geometry is fixed at compile time (TX x TY cells, NCOL = 128 bytes of
// velocity columns), so a thread's column is fixed (threads % NCOL == 0) and
// the job decoding is shifts and masks; only the halo widths are runtime.
template <typename T, int TX, int TY, int SX, int SY, int NT>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 1024 / NT : 1)
    pfc_space_xy_tma_kernel(const __grid_constant__ CUtensorMap tmap, SpaceXYArgs a) {
    constexpr int NCOL = 128 / sizeof(T);
    static_assert(NT % NCOL == 0 && TX % SX == 0 && TY % SY == 0, "tile geometry");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int hx = a.hx, hy = a.hy;
    const int bx = TX + 2 * hx, by = TY + 2 * hy;
    const int sbytes = (int)sizeof(T) * by * bx * NCOL;  // a multiple of 128
    uint64_t* const bar = reinterpret_cast<uint64_t*>(smem_raw);
    T* const sbuf0 = reinterpret_cast<T*>(smem_raw + 128);
    T* const sbuf1 = reinterpret_cast<T*>(smem_raw + 128 + sbytes);
    T* const xs = reinterpret_cast<T*>(smem_raw + 128 + 2 * sbytes);  // [by][TX][NCOL]
    ColStep<T>* const stx = reinterpret_cast<ColStep<T>*>(smem_raw + 128 + 2 * sbytes + sizeof(T) * by * TX * NCOL);
    ColStep<T>* const sty = stx + a.nvx;
    for (int i = threadIdx.x; i < a.nvx + a.nvy; i += NT) {
        if (i < a.nvx) stx[i] = col_step<T>(axis_step<T>(a.vminx, a.dvx, a.cx, i, a.nx, false));
        else sty[i - a.nvx] = col_step<T>(axis_step<T>(a.vminy, a.dvy, a.cy, i - a.nvx, a.ny, a.wall != 0));
    }
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
    }
    __syncthreads();

    const int ntx = a.nx / TX, nty = a.ny / TY;
    const int tiles_per_chunk = ntx * nty;
    const int ntiles = a.nchunks * tiles_per_chunk;  // < 2^31, checked on the host
    const int V = (int)a.V;
    const int c = threadIdx.x % NCOL;  // this thread's velocity column in every job
    const int lane_job = threadIdx.x / NCOL;
    const T* __restrict__ fin = reinterpret_cast<const T*>(a.f_in);
    T* __restrict__ fout = reinterpret_cast<T*>(a.f_out);
    auto issue = [&](int t, int b) {  // one thread
        const int chunk = fdiv(t, a.div_tpc), rem = t - chunk * tiles_per_chunk;
        const int tiy = fdiv(rem, a.div_ntx), tix = rem - tiy * ntx;
        mbar_expect_tx(&bar[b], (uint32_t)sbytes);
        tma_load_3d(b ? sbuf1 : sbuf0, &tmap, chunk * NCOL, tix * TX - hx, tiy * TY - hy, &bar[b]);
    };
    // copies are issued two tiles ahead; bit b of pending: a copy into
    // buffer b has been issued and not yet waited for (uniform over the CTA);
    // bit b of parity: the phase of mbarrier b to wait for
    int t = blockIdx.x;
    unsigned pending = (t < ntiles ? 1u : 0u) | (t + (int)gridDim.x < ntiles ? 2u : 0u);
    if (threadIdx.x == 0) {
        if (pending & 1u) issue(t, 0);
        if (pending & 2u) issue(t + gridDim.x, 1);
    }
    unsigned parity = 0u;
    bool lost = false;
    for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
        const int b = it & 1;
        T* const S = b ? sbuf1 : sbuf0;
        const int chunk = fdiv(t, a.div_tpc), rem = t - chunk * tiles_per_chunk;
        const int tiy = fdiv(rem, a.div_ntx), tix = rem - tiy * ntx;
        const int x0 = tix * TX, y0 = tiy * TY;
        const int vi = chunk * NCOL + c;
        const bool col_ok = vi < V;
        // velocity indices of this thread's column: vi = (iz nvy + iy) nvx + ix
        const int iyz = fdiv(col_ok ? vi : 0, a.div_nvx);
        const int ix = (col_ok ? vi : 0) - iyz * a.nvx;
        const int iz = fdiv(iyz, a.div_nvy);
        const int iy = iyz - iz * a.nvy;
        const ColStep<T> sx = stx[ix];
        const ColStep<T> sy = sty[iy];
        if (!__syncthreads_and(tc::mbar_wait(&bar[b], (parity >> b) & 1u, kCopyWaitPolls))) {
            lost = true;
            break;
        }
        parity ^= 1u << b;
        pending &= ~(1u << b);
        // cells outside the domain (the tensor copy filled them with zeros):
        // rows r < ylo or r >= yhi whole, and in the rows between them the
        // columns xl < xlo or xl >= xhi
        const int xlo = max(0, hx - x0), xhi = min(bx, a.nx - x0 + hx);
        const int ylo = max(0, hy - y0), yhi = min(by, a.ny - y0 + hy);
        if (xlo > 0 || xhi < bx || ylo > 0 || yhi < by) {
            // beyond a wall: the mirror row in the v_y-mirrored column (the
            // velocity box is symmetric in v_y); periodic: the image row
            const int vim = (iz * a.nvy + (a.nvy - 1 - iy)) * a.nvx + ix;
            if (col_ok) {
                // cells to patch: the nyo whole rows outside (nyo * bx cells),
                // then for each of the nin rows inside 8 slots: columns
                // 0..3 (valid below xlo) and xhi + 0..3 (valid below bx)
                const int nyo = ylo + (by - yhi), nin = yhi - ylo;
                const int n_rows = nyo * bx, n_all = n_rows + nin * 8;
                constexpr int L = NT / NCOL, K = 4;
                for (int base = lane_job; base < n_all; base += K * L) {
                    T v[K];
                    int dst[K];
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const int e = base + k * L;
                        dst[k] = -1;
                        int r, xl;
                        if (e < n_rows) {
                            const int ri = fdiv(e, a.div_bx);
                            xl = e - ri * bx;
                            r = ri < ylo ? ri : ri + nin;
                        } else if (e < n_all) {
                            const int j = (e - n_rows) & 7;
                            r = ylo + ((e - n_rows) >> 3);
                            xl = j < 4 ? j : xhi + j - 4;
                            if (j < 4 ? j >= xlo : xl >= bx) continue;
                        } else {
                            continue;
                        }
                        const int gy = y0 - hy + r;
                        int sy_ = gy, svi = vi;
                        if (gy < 0 || gy >= a.ny) {
                            if (a.wall) {
                                sy_ = gy < 0 ? -1 - gy : 2 * a.ny - 1 - gy;
                                svi = vim;
                            } else {
                                sy_ = gy < 0 ? gy + a.ny : gy - a.ny;  // hy <= ny
                            }
                        }
                        int gx = x0 - hx + xl;
                        gx = gx < 0 ? gx + a.nx : (gx >= a.nx ? gx - a.nx : gx);  // hx <= TX <= nx
                        v[k] = fin[((long long)sy_ * a.nx + gx) * V + svi];
                        dst[k] = (r * bx + xl) * NCOL + c;
                    }
#pragma unroll
                    for (int k = 0; k < K; ++k)
                        if (dst[k] >= 0) S[dst[k]] = v[k];
                }
            }
            __syncthreads();
        }
        // phase X: x-advected rows y0 - hy .. y0 + TY + hy - 1 into xs
        if (col_ok) {
            constexpr int NSX = TX / SX;
            for (int jr = lane_job; jr < by * NSX; jr += NT / NCOL) {
                const int seg = jr % NSX, r = jr / NSX;
                const int xs0 = seg * SX;
                const T* src = S + (r * bx + hx + xs0 + sx.off) * NCOL + c;
                T w[SX + 4];
#pragma unroll
                for (int q = 0; q < SX + 4; ++q) w[q] = src[q * NCOL];
                T out[SX];
                pfc_window<T, SX>(sx, w, out);
                T* dst = xs + (r * TX + xs0) * NCOL + c;
#pragma unroll
                for (int k = 0; k < SX; ++k) dst[k * NCOL] = out[k];
            }
        }
        __syncthreads();
        // buffer b is free again: copy the tile two steps ahead into it
        const int tn = t + 2 * (int)gridDim.x;
        if (tn < ntiles) {
            pending |= 1u << b;
            if (threadIdx.x == 0) {
                tc::fence_async_smem();  // order this CTA's reads and patch writes of b before the copy
                issue(tn, b);
            }
        }
        // phase Y: every (x, column) line of xs along y, written to f_out
        if (col_ok) {
            constexpr int NSY = TY / SY;
            const long long ostride = (long long)a.nx * V;
            for (int jx = lane_job; jx < TX * NSY; jx += NT / NCOL) {
                const int xx = jx % TX, seg = jx / TX;
                const int ys0 = seg * SY;
                const T* src = xs + ((hy + ys0 + sy.off) * TX + xx) * NCOL + c;
                T w[SY + 4];
#pragma unroll
                for (int q = 0; q < SY + 4; ++q) w[q] = src[q * TX * NCOL];
                T out[SY];
                pfc_window<T, SY>(sy, w, out);
                T* o = fout + ((long long)(y0 + ys0) * a.nx + x0 + xx) * V + vi;
#pragma unroll
                for (int k = 0; k < SY; ++k) {
                    *o = out[k];
                    o += ostride;
                }
            }
        }
        __syncthreads();  // xs is rewritten by the next tile
    }
    if (lost) {
        // record the loss, then let the copies still in flight land before the
        // CTA's shared memory goes away (bounded as well)
        if (threadIdx.x == 0) {
            atomicAdd(&a.counters[CNT_COPY_TIMEOUT], 1ull);
            for (int b = 0; b < 2; ++b)
                if ((pending >> b) & 1u) tc::mbar_wait(&bar[b], (parity >> b) & 1u, kCopyWaitPolls);
        }
        __syncthreads();
    }
}

size_t pfc_space_xy_smem(const SpaceXYArgs& a, int precision) {
    const size_t es = precision == 64 ? sizeof(double) : sizeof(float);
    const size_t step = precision == 64 ? sizeof(AxisStep<double>) : sizeof(AxisStep<float>);
    return es * (size_t)(a.ty + 2 * a.hy) * a.tx * a.ncol + step * (size_t)(a.nvx + a.nvy);
}

static size_t tma_smem(const SpaceXYArgs& a, int precision) {
    const size_t es = precision == 64 ? sizeof(double) : sizeof(float);
    const size_t step = precision == 64 ? sizeof(AxisStep<double>) : sizeof(AxisStep<float>);
    const size_t box = es * (size_t)(a.ty + 2 * a.hy) * (a.tx + 2 * a.hx) * a.ncol;
    return 128 + 2 * box + es * (size_t)(a.ty + 2 * a.hy) * a.tx * a.ncol + step * (size_t)(a.nvx + a.nvy);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
    static const EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (EncodeTiledFn) nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// f_in as a 3D tensor (velocity index, x, y) with the tile's input box
static bool make_box_map(const SpaceXYArgs& a, int precision, CUtensorMap* m) {
    const EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t es = precision == 64 ? 8 : 4;
    const cuuint64_t dims[3] = {(cuuint64_t)a.V, (cuuint64_t)a.nx, (cuuint64_t)a.ny};
    const cuuint64_t strides[2] = {(cuuint64_t)a.V * es, (cuuint64_t)a.V * es * a.nx};
    const cuuint32_t box[3] = {(cuuint32_t)a.ncol, (cuuint32_t)(a.tx + 2 * a.hx), (cuuint32_t)(a.ty + 2 * a.hy)};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, precision == 64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
              const_cast<void*>(a.f_in), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static int g_xy_sms = 0;

template <typename T, int TX, int TY, int SX, int SY, int NT>
static cudaError_t launch_tma(const CUtensorMap& m, const SpaceXYArgs& a, size_t smem, long long ntiles, cudaStream_t st) {
    auto* k = pfc_space_xy_tma_kernel<T, TX, TY, SX, SY, NT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (g_xy_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_xy_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_xy_sms <= 0) g_xy_sms = 148;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, smem);
    if (per_sm < 1) per_sm = 1;
    long long grid = (long long)g_xy_sms * per_sm;  // persistent
    if (grid > ntiles) grid = ntiles;
    k<<<(unsigned)grid, NT, smem, st>>>(m, a);
    count_launch();
    return cudaGetLastError();
}

template <typename T, int SEG>
static cudaError_t launch_xy(const SpaceXYArgs& a, size_t smem, long long ntiles, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(pfc_space_xy_kernel<T, SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    pfc_space_xy_kernel<T, SEG><<<(unsigned)ntiles, 512, smem, st>>>(a);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_pfc_space_xy(const SpaceXYArgs& args, int precision, cudaStream_t st) {
    // TMA path: 32 x 8 tiles, shifts of at most 2 cells, a 16-byte aligned
    // f_in whose rows are whole multiples of 16 bytes
    {
        SpaceXYArgs a = args;
        a.tx = VL_XY_TX;
        a.ty = VL_XY_TY;
        a.div_nvx = make_fastdiv(a.nvx);
        a.div_nvy = make_fastdiv(a.nvy);
        a.div_ntx = make_fastdiv(a.nx / a.tx > 0 ? a.nx / a.tx : 1);
        a.div_bx = make_fastdiv(a.tx + 2 * a.hx);
        a.div_tpc = make_fastdiv((a.nx / a.tx) * (a.ny / a.ty) > 0 ? (a.nx / a.tx) * (a.ny / a.ty) : 1);
        const size_t es = precision == 64 ? 8 : 4;
        const bool fits = a.hx <= 4 && a.hy <= 4 && a.nx % a.tx == 0 && a.ny % a.ty == 0 && a.hy <= a.ny &&
                          a.ncol * es == 128 && (a.ncol & (a.ncol - 1)) == 0 && (a.V * es) % 16 == 0 &&
                          reinterpret_cast<uintptr_t>(a.f_in) % 16 == 0 && a.counters != nullptr;
        CUtensorMap m;
        if (fits && make_box_map(a, precision, &m)) {
            const size_t smem = tma_smem(a, precision);
            const long long ntiles = (long long)a.nchunks * (a.nx / a.tx) * (a.ny / a.ty);
            if (smem <= 227 * 1024 && ntiles < (1LL << 31) - (1LL << 20) && a.V < (1LL << 31)) {
                constexpr int SX = VL_XY_TX < 16 ? VL_XY_TX : 16, SY = VL_XY_TY < 8 ? VL_XY_TY : 8;
                if (precision == 64) return launch_tma<double, VL_XY_TX, VL_XY_TY, SX, SY, 512>(m, a, smem, ntiles, st);
                return launch_tma<float, VL_XY_TX, VL_XY_TY, SX, SY, VL_XY_NT>(m, a, smem, ntiles, st);
            }
        }
    }
    const size_t smem = pfc_space_xy_smem(args, precision);
    const long long ntiles = (long long)args.nchunks * (args.nx / args.tx) * (args.ny / args.ty);
    const bool seg16 = args.tx % 16 == 0 && args.ty % 16 == 0;
    if (precision == 64)
        return seg16 ? launch_xy<double, 16>(args, smem, ntiles, st) : launch_xy<double, 8>(args, smem, ntiles, st);
    return seg16 ? launch_xy<float, 16>(args, smem, ntiles, st) : launch_xy<float, 8>(args, smem, ntiles, st);
}

}  // namespace vl
