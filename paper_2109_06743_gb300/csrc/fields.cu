// Field solvers (paper Sec. 2.1: FDTD/Yee for Maxwell's equations, two half
// steps per time step in Algorithm 1; Sec. 3.3: conducting walls in y;
// Sec. 3.1: Poisson solver for the electrostatic runs).
//
// Yee staggering on cell (i, j) = [x_i, x_i+1] x [y_j, y_j+1]:
//   Ex(i+1/2, j), Ey(i, j+1/2), Ez(i, j), Bx(i, j+1/2), By(i+1/2, j),
//   Bz(i+1/2, j+1/2); each plane is stored as [ny+1][nx]. In the normalised
// units mu0 = 1 and eps0 = 1/c^2, so dE/dt = c^2 (curl B - J), dB/dt = -curl E.
// One field step of length h is the leapfrog B(h/2), E(h), B(h/2). The current
// is cell centred and averaged to the E positions.
#include "common.cuh"
#include "kernels.cuh"

namespace vl {

enum { EX = 0, EY = 1, EZ = 2, BX = 3, BY = 4, BZ = 5 };

__device__ __forceinline__ int wrapx(int i, int nx) {
    i %= nx;
    return i < 0 ? i + nx : i;
}
// row of a j+1/2 plane; periodic wrap without walls
__device__ __forceinline__ int wrap_half(int j, int ny, int wall) {
    if (wall) return j;
    j %= ny;
    return j < 0 ? j + ny : j;
}

struct Yee {
    double* p;
    int nx, ny;
    long long plane;
    __device__ double& at(int comp, int i, int j) const {
        return p[comp * plane + (long long)j * nx + wrapx(i, nx)];
    }
};

__global__ void faraday_kernel(FieldArgs a, double h) {
    long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    if (id >= (long long)(ny + 1) * nx) return;
    const int i = (int)(id % nx), j = (int)(id / nx);
    Yee y{a.yee, nx, ny, (long long)(ny + 1) * nx};
    const int jp = a.wall ? j + 1 : wrap_half(j + 1, ny, 0);
    if (j < ny) {
        // Bx(i, j+1/2) -= h dEz/dy ; Bz(i+1/2, j+1/2) -= h (dEy/dx - dEx/dy)
        y.at(BX, i, j) -= h * (y.at(EZ, i, jp) - y.at(EZ, i, j)) / a.dy;
        y.at(BZ, i, j) -= h * ((y.at(EY, i + 1, j) - y.at(EY, i, j)) / a.dx -
                               (y.at(EX, i, jp) - y.at(EX, i, j)) / a.dy);
    }
    // By(i+1/2, j) += h dEz/dx on rows 0..ny (walls) or 0..ny-1 (periodic)
    if (a.wall ? j <= ny : j < ny) y.at(BY, i, j) += h * (y.at(EZ, i + 1, j) - y.at(EZ, i, j)) / a.dx;
}

// periodic y: keep row ny of the integer-j planes equal to row 0
__global__ void copy_row_kernel(FieldArgs a, int comp) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.nx) return;
    long long plane = (long long)(a.ny + 1) * a.nx;
    a.yee[comp * plane + (long long)a.ny * a.nx + i] = a.yee[comp * plane + i];
}

__global__ void ampere_kernel(FieldArgs a) {
    long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    if (id >= (long long)(ny + 1) * nx) return;
    const int i = (int)(id % nx), j = (int)(id / nx);
    Yee y{a.yee, nx, ny, (long long)(ny + 1) * nx};
    const double* J = a.cur;
    const double hc2 = a.h * a.c2;
    auto jc = [&](int ii, int jj, int comp) -> double {
        return J[((long long)wrap_half(jj, ny, a.wall) * nx + wrapx(ii, nx)) * 3 + comp];
    };
    const bool interior_int = a.wall ? (j >= 1 && j <= ny - 1) : (j < ny);
    if (interior_int) {
        const int jm = wrap_half(j - 1, ny, a.wall);
        // Ex(i+1/2, j) += h c^2 (dBz/dy - Jx); Jx averaged over cells (i, j-1), (i, j)
        double jx = 0.5 * (jc(i, j - 1, 0) + jc(i, j, 0));
        y.at(EX, i, j) += hc2 * ((y.at(BZ, i, j) - y.at(BZ, i, jm)) / a.dy - jx);
        // Ez(i, j) += h c^2 (dBy/dx - dBx/dy - Jz); Jz over the four cells
        double jz = 0.25 * (jc(i - 1, j - 1, 2) + jc(i, j - 1, 2) + jc(i - 1, j, 2) + jc(i, j, 2));
        y.at(EZ, i, j) += hc2 * ((y.at(BY, i, j) - y.at(BY, i - 1, j)) / a.dx -
                                 (y.at(BX, i, j) - y.at(BX, i, jm)) / a.dy - jz);
    }
    if (j < ny) {
        // Ey(i, j+1/2) += h c^2 (-dBz/dx - Jy); Jy over cells (i-1, j), (i, j)
        double jy = 0.5 * (jc(i - 1, j, 1) + jc(i, j, 1));
        y.at(EY, i, j) += hc2 * (-(y.at(BZ, i, j) - y.at(BZ, i - 1, j)) / a.dx - jy);
    }
}

__global__ void wall_zero_kernel(FieldArgs a) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.nx) return;
    long long plane = (long long)(a.ny + 1) * a.nx;
    a.yee[EX * plane + i] = 0.0;
    a.yee[EX * plane + (long long)a.ny * a.nx + i] = 0.0;
    a.yee[EZ * plane + i] = 0.0;
    a.yee[EZ * plane + (long long)a.ny * a.nx + i] = 0.0;
}

__global__ void centres_kernel(FieldArgs a) {
    long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    if (id >= (long long)ny * nx) return;
    const int i = (int)(id % nx), j = (int)(id / nx);
    Yee y{a.yee, nx, ny, (long long)(ny + 1) * nx};
    double* o = a.eb + id * 6;
    o[0] = 0.5 * (y.at(EX, i, j) + y.at(EX, i, j + 1));
    o[1] = 0.5 * (y.at(EY, i, j) + y.at(EY, i + 1, j));
    o[2] = 0.25 * (y.at(EZ, i, j) + y.at(EZ, i + 1, j) + y.at(EZ, i, j + 1) + y.at(EZ, i + 1, j + 1));
    o[3] = 0.5 * (y.at(BX, i, j) + y.at(BX, i + 1, j));
    o[4] = 0.5 * (y.at(BY, i, j) + y.at(BY, i, j + 1));
    o[5] = y.at(BZ, i, j);
}

cudaError_t launch_maxwell(const FieldArgs& a, cudaStream_t st) {
    long long npts = (long long)(a.ny + 1) * a.nx;
    const int th = 256;
    unsigned g = (unsigned)((npts + th - 1) / th);
    unsigned gx = (unsigned)((a.nx + th - 1) / th);
    int n = 0;
    auto fixup_b = [&]() {
        if (!a.wall) {
            copy_row_kernel<<<gx, th, 0, st>>>(a, BY);
            ++n;
        }
    };
    auto fixup_e = [&]() {
        if (a.wall) {
            wall_zero_kernel<<<gx, th, 0, st>>>(a);
        } else {
            copy_row_kernel<<<gx, th, 0, st>>>(a, EX);
            copy_row_kernel<<<gx, th, 0, st>>>(a, EZ);
            ++n;
        }
        ++n;
    };
    faraday_kernel<<<g, th, 0, st>>>(a, 0.5 * a.h);
    ++n;
    fixup_b();
    ampere_kernel<<<g, th, 0, st>>>(a);
    ++n;
    fixup_e();
    faraday_kernel<<<g, th, 0, st>>>(a, 0.5 * a.h);
    ++n;
    fixup_b();
    unsigned gc = (unsigned)(((long long)a.ny * a.nx + th - 1) / th);
    centres_kernel<<<gc, th, 0, st>>>(a);
    ++n;
    count_launch(n);
    return cudaGetLastError();
}

// J (2D3V, [ncell][3]) = sum_s q_s * src_s[c * stride + off + a], or the
// charge density (1D1V, [ncell]) = bg + sum_s q_s * src_s[c * stride + off]
struct CurrentArgs {
    const double* src[kMaxSpecies];
    double q[kMaxSpecies];
    int nspecies, stride, off, ncomp;
    double bg;
    double* out;
    long long ncell;
};

__global__ void current_kernel(CurrentArgs a) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= a.ncell) return;
    for (int k = 0; k < a.ncomp; ++k) {
        double s = a.ncomp == 1 ? a.bg : 0.0;
        for (int sp = 0; sp < a.nspecies; ++sp) s += a.q[sp] * a.src[sp][c * a.stride + a.off + k];
        a.out[c * a.ncomp + k] = s;
    }
}

cudaError_t launch_current(double* cur, const double* const* src, const double* q, int nspecies, int stride,
                           int off, long long ncell, int nvdim, double bg, cudaStream_t st) {
    CurrentArgs a;
    for (int s = 0; s < nspecies; ++s) {
        a.src[s] = src[s];
        a.q[s] = q[s];
    }
    a.nspecies = nspecies;
    a.stride = stride;
    a.off = off;
    a.ncomp = nvdim == 1 ? 1 : 3;
    a.bg = bg;
    a.out = cur;
    a.ncell = ncell;
    current_kernel<<<(unsigned)((ncell + 127) / 128), 128, 0, st>>>(a);
    count_launch();
    return cudaGetLastError();
}

// 1D periodic Poisson dE/dx = rho: face values by a running sum, zero mean,
// then cell centres as the average of the two faces. One warp: each lane
// sums a contiguous run of cells, an inclusive scan over the lanes gives each
// run's starting face value, and the mean is a warp sum.
__global__ void poisson_kernel(const double* rho, double* eb, int nx, double dx) {
    constexpr unsigned kAll = 0xffffffffu;
    if (blockIdx.x != 0) return;
    const int lane = threadIdx.x & 31;
    const int per = (nx + 31) / 32, lo = min(lane * per, nx), hi = min(lo + per, nx);
    double loc = 0.0;
    for (int i = lo; i < hi; ++i) loc += dx * rho[i];
    double inc = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double t = __shfl_up_sync(kAll, inc, o);
        if (lane >= o) inc += t;
    }
    const double before = inc - loc;  // running sum up to the face below lo
    const double total = __shfl_sync(kAll, inc, 31);
    double msum = 0.0, acc = before;
    for (int i = lo; i < hi; ++i) {
        acc += dx * rho[i];
        msum += acc;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) msum += __shfl_xor_sync(kAll, msum, o);
    const double mean = msum / nx;
    // face -1/2 equals face nx-1/2 (periodic)
    double prev = (lane == 0 ? total : before) - mean;
    acc = before;
    for (int i = lo; i < hi; ++i) {
        acc += dx * rho[i];
        const double face = acc - mean;
        eb[(long long)i * 6] = 0.5 * (prev + face);
        prev = face;
    }
}

cudaError_t launch_poisson(const double* rho, double* eb, int nx, double dx, cudaStream_t st) {
    poisson_kernel<<<1, 32, 0, st>>>(rho, eb, nx, dx);
    count_launch();
    return cudaGetLastError();
}

}  // namespace vl
