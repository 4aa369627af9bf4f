// Ten-moment fluid step (paper Sec. 2.1 equations with the third moment from
// f, Sec. 2.2; CWENO of Kurganov and Levy 2000 and SSP-RK3 of Shu and Osher
// 1988, cited in Sec. 2.1). With FluidArgs.closure the same kernel runs the
// stand-alone fluid model of Sec. 2.3 (gradient heat-flux closure).
//
// Per species the state is U = (n, nu_a, E2_ab), E2 = P/m = int v v f. The
// equations divided by m read
//   dn/dt     + d_k nu_k    = 0
//   dnu_a/dt  + d_k E2_ka   = (q/m) (n E_a + (nu x B)_a)
//   dE2_ab/dt + d_k E3_kab  = (q/m) (nu_a E_b + nu_b E_a + C_ab + C_ba),
// C_ab = ((row a of E2) x B)_b, E3 = int v v v f taken from the Vlasov solver
// and reconstructed with the same CWENO polynomials as U. Fluxes are the
// central-upwind (local Lax-Friedrichs) flux with the ten-moment wave speed
// |u_d| + sqrt(3 Theta_dd) of the two neighbouring cells. One thread per cell
// and stage. The state stays in FP64; the reconstruction, fluxes and sources
// (the right-hand side L) are computed in R = double in FP64 mode and in
// R = float in FP32 mode (on GB300 the FP64 pipe runs at ~1/58 of the FP32
// pipe), and the Runge-Kutta combination U0 + dt L is formed in FP64.
#include "common.cuh"
#include "kernels.cuh"

namespace vl {

__device__ __forceinline__ int s2(int a, int b) {
    return a == 0 ? b : (a == 1 ? (b == 0 ? 1 : b + 2) : (b == 0 ? 2 : (b == 1 ? 4 : 5)));
}

// index of the symmetric triple in xxx,xxy,xxz,xyy,xyz,xzz,yyy,yyz,yzz,zzz
__device__ __forceinline__ int s3(int a, int b, int c) {
    int x = (a == 0) + (b == 0) + (c == 0), y = (a == 1) + (b == 1) + (c == 1);
    // by number of x, then y
    if (x == 3) return 0;
    if (x == 2) return y == 1 ? 1 : 2;
    if (x == 1) return y == 2 ? 3 : (y == 1 ? 4 : 5);
    return y == 3 ? 6 : (y == 2 ? 7 : (y == 1 ? 8 : 9));
}

template <typename R>
__device__ __forceinline__ void cweno3_point(R um, R u0, R up, R* left, R* right) {
    const R eps = R(1e-6);
    R il = (u0 - um) * (u0 - um), ir = (up - u0) * (up - u0);
    R d2 = up - R(2) * u0 + um, d1 = up - um;
    R ic = (R(13) / R(3)) * d2 * d2 + R(0.25) * d1 * d1;
    R al = R(0.25) / ((eps + il) * (eps + il));
    R ar = R(0.25) / ((eps + ir) * (eps + ir));
    R ac = R(0.5) / ((eps + ic) * (eps + ic));
    R inv = R(1) / (al + ar + ac);
    R wl = al * inv, wr = ar * inv, wc = ac * inv;
    // values at xi = -1/2 and +1/2 of the linear left/right and the central
    // polynomial P_C = (P_opt - P_L/4 - P_R/4) / (1/2)
    R base = u0 - d2 / R(24) + R(0.125) * d2;
    R optl = base - R(0.25) * d1, optr = base + R(0.25) * d1;
    R ll = u0 - R(0.5) * (u0 - um), lr = u0 + R(0.5) * (u0 - um);
    R rl = u0 - R(0.5) * (up - u0), rr = u0 + R(0.5) * (up - u0);
    R cl = R(2) * optl - R(0.5) * ll - R(0.5) * rl;
    R cr = R(2) * optr - R(0.5) * lr - R(0.5) * rr;
    *left = wl * ll + wr * rl + wc * cl;
    *right = wl * lr + wr * rr + wc * cr;
}

struct FluidCtx {
    const FluidArgs* a;
    int nc, nq, qoff;
    bool use0, use1;  // wq0 != 0, wq1 != 0 (decided once per thread)
};

// sign of a component under y -> -y (v_y -> -v_y)
__device__ __forceinline__ double parity_state(int k) {
    // n nux nuy nuz xx xy xz yy yz zz
    return (k == 2 || k == 5 || k == 8) ? -1.0 : 1.0;
}
__device__ __forceinline__ double parity_q(int k) {
    // xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz
    return (k == 1 || k == 4 || k == 6 || k == 8) ? -1.0 : 1.0;
}

// resolve (ix, iy) with periodic x and periodic-or-wall y; returns the
// linear cell index and the mirror flag
__device__ __forceinline__ long long resolve(const FluidArgs& a, int ix, int iy, bool* mir) {
    ix %= a.nx;
    if (ix < 0) ix += a.nx;
    *mir = false;
    if (iy < 0 || iy >= a.ny) {
        if (a.bc_y == 1) {
            iy = iy < 0 ? -1 - iy : 2 * a.ny - 1 - iy;
            *mir = true;
        } else {
            iy %= a.ny;
            if (iy < 0) iy += a.ny;
        }
    }
    return (long long)iy * a.nx + ix;
}

// In FP32 mode the stage input and the weighted third moments are converted
// to float once per stage (fluid_prep_kernel) instead of at each of the ~16
// stencil reads of every value (FP64-to-FP32 conversions run on the FP64
// pipe); the values are the same.
template <typename R>
__device__ __forceinline__ R state_at(const FluidCtx& c, int k, int ix, int iy) {
    bool mir;
    long long id = resolve(*c.a, ix, iy, &mir);
    R v = (sizeof(R) == 4 && c.a->Usf) ? (R)c.a->Usf[id * c.nc + k] : (R)c.a->Us[id * c.nc + k];
    return (mir && c.a->nvdim == 3) ? v * (R)parity_state(k) : v;
}

// Q = wq0 q0 + wq1 q1 (the weights are 0, 1/2 or 1, exact in R)
template <typename R>
__device__ __forceinline__ R q_value(const FluidArgs& a, const FluidCtx& c, long long id, int k) {
    R v = R(0);
    if (c.use0) v += (R)a.wq0 * (R)a.q0[id * a.nmom + c.qoff + k];
    if (c.use1) v += (R)a.wq1 * (R)a.q1[id * a.nmom + c.qoff + k];
    return v;
}

template <typename R>
__device__ __forceinline__ R q_at(const FluidCtx& c, int k, int ix, int iy) {
    bool mir;
    long long id = resolve(*c.a, ix, iy, &mir);
    const FluidArgs& a = *c.a;
    const R v = (sizeof(R) == 4 && a.Qf) ? (R)a.Qf[id * c.nq + k] : q_value<R>(a, c, id, k);
    return (mir && a.nvdim == 3) ? v * (R)parity_q(k) : v;
}

template <typename R>
__device__ __forceinline__ R wave_speed(int nvdim, int dir, const R* u) {
    R n = u[0];
    if (!(n > R(0))) return R(0);
    R ud = u[1 + dir] / n;
    R e2 = nvdim == 1 ? u[2] : u[4 + s2(dir, dir)];
    R th = e2 / n - ud * ud;
    if (th < R(0)) th = R(0);
    return fabs(ud) + sqrt(R(3) * th);
}

template <typename R>
__device__ __forceinline__ R flux_of(int nvdim, int dir, int k, const R* u, const R* q) {
    if (nvdim == 1) return k == 0 ? u[1] : (k == 1 ? u[2] : q[0]);
    if (k == 0) return u[1 + dir];
    if (k < 4) return u[4 + s2(dir, k - 1)];
    const int ab[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    return q[s3(dir, ab[k - 4][0], ab[k - 4][1])];
}

// Gradient-closure model (Sec. 2.3): with zero heat flux the third moment
// is that of the Maxwellian with the state's n, u and E2,
//   E3_kab = u_k E2_ab + u_a E2_kb + u_b E2_ka - 2 n u_k u_a u_b,
// evaluated on the reconstructed interface states.
template <typename R>
__device__ __forceinline__ void closure_e3(const R* s, R* e3) {
    const R n = s[0];
    if (!(n > R(0))) {
#pragma unroll
        for (int k = 0; k < 10; ++k) e3[k] = R(0);
        return;
    }
    const R inv = R(1) / n;
    const R v[3] = {s[1] * inv, s[2] * inv, s[3] * inv};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a; b < 3; ++b)
#pragma unroll
            for (int k = b; k < 3; ++k)
                e3[s3(a, b, k)] = v[k] * s[4 + s2(a, b)] + v[a] * s[4 + s2(k, b)] + v[b] * s[4 + s2(k, a)] -
                                  R(2) * n * v[k] * v[a] * v[b];
}

// theta = E2 / n - u u of cell (ix, iy), ghosts as for the state
template <typename R>
__device__ __forceinline__ void theta_cell(const FluidCtx& c, int ix, int iy, R* th) {
    R s[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) s[k] = state_at<R>(c, k, ix, iy);
    const R n = s[0];
    const R inv = n > R(0) ? R(1) / n : R(0);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a; b < 3; ++b) th[s2(a, b)] = s[4 + s2(a, b)] * inv - (s[1 + a] * inv) * (s[1 + b] * inv);
}

// value of component k of the state (q = false) or of the third moments
// (q = true) in a resolved cell (id, mirror flag)
template <typename R>
__device__ __forceinline__ R value_at(const FluidCtx& c, bool q, int k, long long id, bool mir) {
    const FluidArgs& a = *c.a;
    R v;
    if (!q) v = (sizeof(R) == 4 && a.Usf) ? (R)a.Usf[id * c.nc + k] : (R)a.Us[id * c.nc + k];
    else v = (sizeof(R) == 4 && a.Qf) ? (R)a.Qf[id * c.nq + k] : q_value<R>(a, c, id, k);
    if (mir && a.nvdim == 3) v *= (R)(q ? parity_q(k) : parity_state(k));
    return v;
}

// Numerical fluxes through the two interfaces of a cell in direction dir
// (Hm: with the neighbour below, Hp: with the neighbour above). The five
// cells of the stencil are resolved once; each of the three middle cells is
// reconstructed once (its left and right interface values), which serves
// both interfaces.
// The numerical fluxes of cell_fluxes with the third moments from f (no
// closure), one flux component at a time so that few values are live: the
// interface states of component k (for the dissipation term) and of the
// component whose value is k's flux (state component 1+dir, 4+(dir,k-1) or
// third moment (dir,a,b)). The wave speeds come from the cell averages.
template <typename R, int NV>
__device__ __forceinline__ void cell_fluxes_lean(const FluidCtx& c, int dir, int ix, int iy, R* Hm, R* Hp) {
    constexpr int NC = NV == 1 ? 3 : 10;
    long long id[5];
    bool mir[5];
#pragma unroll
    for (int o = 0; o < 5; ++o)
        id[o] = resolve(*c.a, ix + (dir == 0 ? o - 2 : 0), iy + (dir == 1 ? o - 2 : 0), &mir[o]);
    // wave speeds |u_d| + sqrt(3 Theta_dd) of cells -1, 0, +1
    R ws[3];
    const int kd = NV == 1 ? 2 : 4 + s2(dir, dir);
#pragma unroll
    for (int o = 0; o < 3; ++o) {
        const R n = value_at<R>(c, false, 0, id[o + 1], mir[o + 1]);
        const R nu = value_at<R>(c, false, 1 + dir, id[o + 1], mir[o + 1]);
        const R e2 = value_at<R>(c, false, kd, id[o + 1], mir[o + 1]);
        R w = R(0);
        if (n > R(0)) {
            const R ud = nu / n;
            R th = e2 / n - ud * ud;
            if (th < R(0)) th = R(0);
            w = fabs(ud) + sqrt(R(3) * th);
        }
        ws[o] = w;
    }
    const R sm = fmax(ws[0], ws[1]), sp = fmax(ws[1], ws[2]);
    // interface states of one component: the right value of cell -1, the
    // left and right values of cell 0 and the left value of cell +1
    auto recon = [&](bool q, int k, R& rm, R& l0, R& r0, R& lp) {
        const R a0 = value_at<R>(c, q, k, id[0], mir[0]), a1 = value_at<R>(c, q, k, id[1], mir[1]);
        const R a2 = value_at<R>(c, q, k, id[2], mir[2]), a3 = value_at<R>(c, q, k, id[3], mir[3]);
        const R a4 = value_at<R>(c, q, k, id[4], mir[4]);
        R l, r;
        cweno3_point<R>(a0, a1, a2, &l, &r);
        rm = r;
        cweno3_point<R>(a1, a2, a3, &l0, &r0);
        cweno3_point<R>(a2, a3, a4, &lp, &r);
    };
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        R um, u0, up, cp;
        recon(false, k, um, u0, up, cp);
        // the flux of component k
        bool fq;
        int fk;
        if (NV == 1) {
            fq = k == 2;
            fk = k == 0 ? 1 : (k == 1 ? 2 : 0);
        } else if (k == 0) {
            fq = false;
            fk = 1 + dir;
        } else if (k < 4) {
            fq = false;
            fk = 4 + s2(dir, k - 1);
        } else {
            const int ab[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
            fq = true;
            fk = s3(dir, ab[k - 4][0], ab[k - 4][1]);
        }
        R fm, f0, fp, fc;
        recon(fq, fk, fm, f0, fp, fc);
        Hm[k] = R(0.5) * (fm + f0) - R(0.5) * sm * (u0 - um);
        Hp[k] = R(0.5) * (fp + fc) - R(0.5) * sp * (cp - up);
    }
}

template <typename R, int NV>
__device__ __forceinline__ void cell_fluxes(const FluidCtx& c, int dir, int ix, int iy, R* Hm, R* Hp) {
    constexpr int NC = NV == 1 ? 3 : 10, NQ = NV == 1 ? 1 : 10;
    long long id[5];
    bool mir[5];
#pragma unroll
    for (int o = 0; o < 5; ++o)
        id[o] = resolve(*c.a, ix + (dir == 0 ? o - 2 : 0), iy + (dir == 1 ? o - 2 : 0), &mir[o]);
    // uE[p][side]: reconstruction in cell p-1 (p = 0, 1, 2 for cells -1, 0, +1)
    R um[10], u0[10], up[10], cm[10], c0[10], cp[10];  // left/right states of the two interfaces
    R qm_[10], q0_[10], qp_[10], qmm[10];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const R a0 = value_at<R>(c, false, k, id[0], mir[0]), a1 = value_at<R>(c, false, k, id[1], mir[1]);
        const R a2 = value_at<R>(c, false, k, id[2], mir[2]), a3 = value_at<R>(c, false, k, id[3], mir[3]);
        const R a4 = value_at<R>(c, false, k, id[4], mir[4]);
        R l, r;
        cweno3_point<R>(a0, a1, a2, &l, &r);  // cell -1
        um[k] = r;                            // left state of the lower interface
        cweno3_point<R>(a1, a2, a3, &l, &r);  // cell 0
        u0[k] = l;                            // right state of the lower interface
        up[k] = r;                            // left state of the upper interface
        cweno3_point<R>(a2, a3, a4, &l, &r);  // cell +1
        cp[k] = l;                            // right state of the upper interface
        cm[k] = a1;
        c0[k] = a2;
        qmm[k] = a3;  // cell averages of cell +1 (wave speed)
    }
    if (c.a->closure) {
        closure_e3<R>(um, qm_);
        closure_e3<R>(u0, q0_);
        closure_e3<R>(up, qp_);
    }
    R qcp[10];
    if (c.a->closure) {
        closure_e3<R>(cp, qcp);
    } else {
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            const R a0 = value_at<R>(c, true, k, id[0], mir[0]), a1 = value_at<R>(c, true, k, id[1], mir[1]);
            const R a2 = value_at<R>(c, true, k, id[2], mir[2]), a3 = value_at<R>(c, true, k, id[3], mir[3]);
            const R a4 = value_at<R>(c, true, k, id[4], mir[4]);
            R l, r;
            cweno3_point<R>(a0, a1, a2, &l, &r);
            qm_[k] = r;
            cweno3_point<R>(a1, a2, a3, &l, &r);
            q0_[k] = l;
            qp_[k] = r;
            cweno3_point<R>(a2, a3, a4, &l, &r);
            qcp[k] = l;
        }
    }
    constexpr int nvdim = NV;
    const R sm = fmax(wave_speed<R>(nvdim, dir, cm), wave_speed<R>(nvdim, dir, c0));
    const R sp = fmax(wave_speed<R>(nvdim, dir, c0), wave_speed<R>(nvdim, dir, qmm));
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        Hm[k] = R(0.5) * (flux_of<R>(nvdim, dir, k, um, qm_) + flux_of<R>(nvdim, dir, k, u0, q0_)) -
                R(0.5) * sm * (u0[k] - um[k]);
        Hp[k] = R(0.5) * (flux_of<R>(nvdim, dir, k, up, qp_) + flux_of<R>(nvdim, dir, k, cp, qcp)) -
                R(0.5) * sp * (cp[k] - up[k]);
    }
}

// One thread per cell and stage; NV = 1 (1D1V: three components) or 3
// (2D3V: ten), a compile-time count so that the per-component arrays stay in
// registers.
#ifndef VL_FLUID_MIN_BLOCKS_F32
#define VL_FLUID_MIN_BLOCKS_F32 8
#endif
#ifndef VL_FLUID_MIN_BLOCKS_F64
#define VL_FLUID_MIN_BLOCKS_F64 1
#endif
template <typename R, int NV, bool CLOSURE>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? VL_FLUID_MIN_BLOCKS_F32 : VL_FLUID_MIN_BLOCKS_F64)
    fluid_stage_kernel(FluidArgs a) {
    constexpr int NC = NV == 1 ? 3 : 10;
    long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (cell >= (long long)a.nx * a.ny) return;
    const int ix = (int)(cell % a.nx), iy = (int)(cell / a.nx);
    FluidCtx c;
    c.a = &a;
    c.nc = NC;
    c.nq = NV == 1 ? 1 : 10;
    c.qoff = NV == 1 ? 3 : 10;
    c.use0 = a.wq0 != 0.0;
    c.use1 = a.wq1 != 0.0;
    R L[10];
#pragma unroll
    for (int k = 0; k < NC; ++k) L[k] = R(0);
    constexpr int ndir = NV == 1 ? 1 : 2;
    R Hm[10], Hp[10];
#pragma unroll
    for (int dir = 0; dir < ndir; ++dir) {
        const R invh = (R)(1.0 / (dir == 0 ? a.dx : a.dy));
        if (CLOSURE) cell_fluxes<R, NV>(c, dir, ix, iy, Hm, Hp);
        else cell_fluxes_lean<R, NV>(c, dir, ix, iy, Hm, Hp);
        // walls: the interface beyond the last row is the wall itself
        // (mirror ghosts already give its flux); nothing special needed
#pragma unroll
        for (int k = 0; k < NC; ++k) L[k] -= (Hp[k] - Hm[k]) * invh;
    }
    R u[10], eb[6];
#pragma unroll
    for (int k = 0; k < NC; ++k) u[k] = (R)a.Us[cell * NC + k];
#pragma unroll
    for (int k = 0; k < 6; ++k) eb[k] = (R)a.eb[cell * 6 + k];
    const R qm = (R)a.qm;
    if (NV == 1) {
        L[1] += qm * u[0] * eb[0];
        L[2] += qm * R(2) * u[1] * eb[0];
    } else {
        const R* E = eb;
        const R* B = eb + 3;
        const R* nu = u + 1;
        L[1] += qm * (u[0] * E[0] + nu[1] * B[2] - nu[2] * B[1]);
        L[2] += qm * (u[0] * E[1] + nu[2] * B[0] - nu[0] * B[2]);
        L[3] += qm * (u[0] * E[2] + nu[0] * B[1] - nu[1] * B[0]);
        R M[3][3];
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) M[p][q] = u[4 + s2(p, q)];
        R C[3][3];
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            C[p][0] = M[p][1] * B[2] - M[p][2] * B[1];
            C[p][1] = M[p][2] * B[0] - M[p][0] * B[2];
            C[p][2] = M[p][0] * B[1] - M[p][1] * B[0];
        }
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = p; q < 3; ++q) L[4 + s2(p, q)] += qm * (nu[p] * E[q] + nu[q] * E[p] + C[p][q] + C[q][p]);
        if (CLOSURE) {
            // heat flux of the closure: -(1/m) div Q = chi_k0 n v_t lap theta,
            // v_t = sqrt(tr(theta) / 3), five-point Laplacian
            R t0[6], tw[6], te[6], ts[6], tn[6];
            theta_cell<R>(c, ix, iy, t0);
            theta_cell<R>(c, ix - 1, iy, tw);
            theta_cell<R>(c, ix + 1, iy, te);
            theta_cell<R>(c, ix, iy - 1, ts);
            theta_cell<R>(c, ix, iy + 1, tn);
            const R tr = t0[0] + t0[3] + t0[5];
            const R vt = sqrt(tr > R(0) ? tr / R(3) : R(0));
            const R coef = (R)a.chi_k0 * u[0] * vt;
            const R ix2 = (R)(1.0 / (a.dx * a.dx)), iy2 = (R)(1.0 / (a.dy * a.dy));
#pragma unroll
            for (int k = 0; k < 6; ++k)
                L[4 + k] += coef * ((te[k] - R(2) * t0[k] + tw[k]) * ix2 + (tn[k] - R(2) * t0[k] + ts[k]) * iy2);
        }
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        double us = a.Us[cell * NC + k];
        double u0 = a.a0 != 0.0 ? a.U0[cell * NC + k] : 0.0;
        a.Uout[cell * NC + k] = a.a0 * u0 + a.a1 * (us + a.dt * (double)L[k]);
    }
}

// FP32 copies of the stage input and of the weighted third moments
__global__ void fluid_prep_kernel(FluidArgs a) {
    long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (cell >= (long long)a.nx * a.ny) return;
    FluidCtx c;
    c.a = &a;
    c.nc = a.nvdim == 1 ? 3 : 10;
    c.nq = a.nvdim == 1 ? 1 : 10;
    c.qoff = a.nvdim == 1 ? 3 : 10;
    c.use0 = a.wq0 != 0.0;
    c.use1 = a.wq1 != 0.0;
    for (int k = 0; k < c.nc; ++k) a.Usf[cell * c.nc + k] = (float)a.Us[cell * c.nc + k];
    if (a.Qf)
        for (int k = 0; k < c.nq; ++k) a.Qf[cell * c.nq + k] = q_value<float>(a, c, cell, k);
}

cudaError_t launch_fluid_stage(const FluidArgs& args, cudaStream_t st) {
    FluidArgs a = args;
    long long n = (long long)a.nx * a.ny;
    int threads = 128;
    if (a.precision == 64) {
        a.Usf = nullptr;
        a.Qf = nullptr;
    }
    if (a.Usf) {
        fluid_prep_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(a);
        count_launch();
    }
    const unsigned grid = (unsigned)((n + threads - 1) / threads);
    if (a.nvdim == 1) {
        if (a.precision == 64) fluid_stage_kernel<double, 1, false><<<grid, threads, 0, st>>>(a);
        else fluid_stage_kernel<float, 1, false><<<grid, threads, 0, st>>>(a);
    } else if (a.closure) {
        if (a.precision == 64) fluid_stage_kernel<double, 3, true><<<grid, threads, 0, st>>>(a);
        else fluid_stage_kernel<float, 3, true><<<grid, threads, 0, st>>>(a);
    } else {
        if (a.precision == 64) fluid_stage_kernel<double, 3, false><<<grid, threads, 0, st>>>(a);
        else fluid_stage_kernel<float, 3, false><<<grid, threads, 0, st>>>(a);
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace vl
