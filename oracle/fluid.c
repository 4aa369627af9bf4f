/*
 * Oracle: ten-moment fluid step (test infrastructure only; see oracle.h).
 *
 * Paper Sec. 2.1 (continuity, momentum and second-moment equations) with the
 * third moment Q taken from f (Sec. 2.2), solved by the semi-discrete central
 * CWENO scheme of Kurganov and Levy (2000) and the SSP Runge-Kutta scheme of
 * Shu and Osher (1988) (Sec. 2.1). Q enters through the flux of the second
 * moment and is reconstructed with the same CWENO polynomials (Sec. 2.2:
 * "incorporated into the CWENO reconstruction"). The RK stages use Q at t,
 * t+dt and t+dt/2 (Algorithm 1) and E, B frozen at t+dt/2.
 *
 * Per species the state is U = (n, nu_a, E2_ab) with E2 = P/m = int v v f;
 * dividing the paper's equations by m gives
 *   dn/dt    + div(nu)  = 0
 *   dnu_a/dt + d_k E2_ka = (q/m) (n E_a + (nu x B)_a)
 *   dE2_ab/dt + d_k E3_kab = (q/m) (nu_a E_b + nu_b E_a + C_ab + C_ba),
 *   C_ab = ((row a of E2) x B)_b.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* index of the symmetric pair (a,b) in xx,xy,xz,yy,yz,zz */
static int sym2(int a, int b) {
    static const int T[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    return T[a][b];
}
/* index of the symmetric triple in xxx,xxy,xxz,xyy,xyz,xzz,yyy,yyz,yzz,zzz */
static int sym3(int a, int b, int c) {
    int s[3] = {a, b, c};
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (s[j] < s[i]) { int t = s[i]; s[i] = s[j]; s[j] = t; }
    static const int T[3][3][3] = {
        {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}},
        {{1, 3, 4}, {3, 6, 7}, {4, 7, 8}},
        {{2, 4, 5}, {4, 7, 8}, {5, 8, 9}}};
    return T[s[0]][s[1]][s[2]];
}

/* CWENO3 reconstruction (Kurganov-Levy 2000) in a cell with averages um, u0,
 * up: point values at the left (xl) and right (xr) cell interfaces. */
static void cweno3(double um, double u0, double up, double* xl, double* xr) {
    const double eps = 1e-6;
    const double cl = 0.25, cr = 0.25, cc = 0.5;
    double isl = (u0 - um) * (u0 - um);
    double isr = (up - u0) * (up - u0);
    double isc = 13.0 / 3.0 * (up - 2.0 * u0 + um) * (up - 2.0 * u0 + um) +
                 0.25 * (up - um) * (up - um);
    double al = cl / ((eps + isl) * (eps + isl));
    double ar = cr / ((eps + isr) * (eps + isr));
    double ac = cc / ((eps + isc) * (eps + isc));
    double s = al + ar + ac;
    double wl = al / s, wr = ar / s, wc = ac / s;
    /* the three polynomials at xi = -1/2 and +1/2 (xi = (x - x_j)/dx) */
    double d2 = up - 2.0 * u0 + um;
    double popt_l = u0 - d2 / 24.0 - 0.25 * (up - um) + 0.125 * d2;
    double popt_r = u0 - d2 / 24.0 + 0.25 * (up - um) + 0.125 * d2;
    double pl_l = u0 - 0.5 * (u0 - um), pl_r = u0 + 0.5 * (u0 - um);
    double pr_l = u0 - 0.5 * (up - u0), pr_r = u0 + 0.5 * (up - u0);
    double pc_l = (popt_l - cl * pl_l - cr * pr_l) / cc;
    double pc_r = (popt_r - cl * pl_r - cr * pr_r) / cc;
    *xl = wl * pl_l + wr * pr_l + wc * pc_l;
    *xr = wl * pl_r + wr * pr_r + wc * pc_r;
}

/* parity of a state component (3V) under y -> -y */
static double parity_u(int comp) {
    static const double P[10] = {1, 1, -1, 1, 1, -1, 1, 1, -1, 1};
    return P[comp];
}
static double parity_q(int comp) {
    static const double P[10] = {1, -1, 1, 1, -1, 1, -1, 1, -1, 1};
    return P[comp];
}

typedef struct {
    const or_grid* g;
    const or_species* sp;
    int ncomp, nq;
} fl_ctx;

/* fetch component comp of cell (ix, iy) of field A (ncomp per cell) with
 * periodic x and periodic-or-wall y ghosts */
static double fetch(const fl_ctx* c, const double* A, int stride, int comp,
                    int ix, int iy, int is_q) {
    const or_grid* g = c->g;
    ix = ((ix % g->nx) + g->nx) % g->nx;
    double sgn = 1.0;
    if (iy < 0 || iy >= g->ny) {
        if (g->bc_y == 1) {
            iy = iy < 0 ? -1 - iy : 2 * g->ny - 1 - iy;
            if (g->nvdim == 3) sgn = is_q ? parity_q(comp) : parity_u(comp);
        } else {
            iy = ((iy % g->ny) + g->ny) % g->ny;
        }
    }
    return sgn * A[((long)iy * g->nx + ix) * stride + comp];
}

static double fetch_state(const fl_ctx* c, const double* U, int comp, int ix, int iy) {
    return fetch(c, U, c->ncomp, comp, ix, iy, 0);
}

/* flux component k (of ncomp) in direction dir from state u and third
 * moments q */
static double flux_comp(int d, int dir, int k, const double* u, const double* q) {
    if (d == 1) {
        if (k == 0) return u[1];
        if (k == 1) return u[2];
        return q[0];
    }
    if (k == 0) return u[1 + dir];
    if (k <= 3) return u[4 + sym2(dir, k - 1)];
    /* k >= 4: E2 component (a,b) */
    static const int AB[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    int a = AB[k - 4][0], b = AB[k - 4][1];
    return q[sym3(dir, a, b)];
}

static double wave_speed(int d, int dir, const double* u) {
    double n = u[0];
    if (!(n > 0.0)) return 0.0;
    double ud = u[1 + dir] / n;
    double e2 = d == 1 ? u[2] : u[4 + sym2(dir, dir)];
    double th = e2 / n - ud * ud;
    if (th < 0.0) th = 0.0;
    return fabs(ud) + sqrt(3.0 * th);
}

/* Gradient-closure model (Sec. 2.3): the third moment E3 = int v v v f of a
 * state with zero heat flux, i.e. of the Maxwellian with the state's n, u
 * and E2:  E3_kab = u_k E2_ab + u_a E2_kb + u_b E2_ka - 2 n u_k u_a u_b
 * (from Q = calQ - sym(u (x) calP) + 2 m n u u u with Q = 0, divided by m).
 * The heat flux itself enters as a source (closure_source). */
static void maxwellian_e3(const double* u, double* e3) {
    double n = u[0];
    if (!(n > 0.0)) {
        for (int k = 0; k < 10; ++k) e3[k] = 0.0;
        return;
    }
    double v[3] = {u[1] / n, u[2] / n, u[3] / n};
    for (int a = 0; a < 3; ++a)
        for (int b = a; b < 3; ++b)
            for (int k = b; k < 3; ++k)
                e3[sym3(a, b, k)] = v[k] * u[4 + sym2(a, b)] + v[a] * u[4 + sym2(k, b)] +
                                    v[b] * u[4 + sym2(k, a)] - 2.0 * n * v[k] * v[a] * v[b];
}

/* temperature per mass of cell (ix, iy) (ghosts resolved like the state):
 * theta_ab = E2_ab / n - u_a u_b */
static void theta_at(const fl_ctx* c, const double* U, int ix, int iy, double* th) {
    double u[10];
    for (int k = 0; k < 10; ++k) u[k] = fetch_state(c, U, k, ix, iy);
    double n = u[0];
    for (int a = 0; a < 3; ++a)
        for (int b = a; b < 3; ++b)
            th[sym2(a, b)] = n > 0.0 ? u[4 + sym2(a, b)] / n - (u[1 + a] / n) * (u[1 + b] / n) : 0.0;
}

/* semi-discrete right-hand side L(U); Q == NULL selects the closure model's
 * Maxwellian third moment, reconstructed state by state */
static void rhs(const fl_ctx* c, const double* U, const double* Q,
                const double* EB, double* out) {
    const or_grid* g = c->g;
    int d = g->nvdim, nc = c->ncomp, nq = c->nq;
    long ncell = (long)g->nx * g->ny;
    double qm = c->sp->q / c->sp->m;
    for (long i = 0; i < ncell * nc; ++i) out[i] = 0.0;
    int ndir = d == 1 ? 1 : 2;
    for (int dir = 0; dir < ndir; ++dir) {
        double h = dir == 0 ? g->dx : g->dy;
        for (int iy = 0; iy < g->ny; ++iy)
            for (int ix = 0; ix < g->nx; ++ix) {
                /* interface between cell L = (ix,iy) and R = +1 along dir;
                 * with walls in y the last interface is the wall itself */
                int lx = ix, ly = iy;
                int rx = dir == 0 ? ix + 1 : ix, ry = dir == 1 ? iy + 1 : iy;
                double uL[10], uR[10], qL[10], qR[10], cL[10], cR[10];
                for (int k = 0; k < nc; ++k) {
                    int ox = dir == 0, oy = dir == 1;
                    double a0 = fetch(c, U, nc, k, lx - ox, ly - oy, 0);
                    double a1 = fetch(c, U, nc, k, lx, ly, 0);
                    double a2 = fetch(c, U, nc, k, rx, ry, 0);
                    double a3 = fetch(c, U, nc, k, rx + ox, ry + oy, 0);
                    double xl, xr;
                    cweno3(a0, a1, a2, &xl, &xr);
                    uL[k] = xr; /* right edge of the left cell */
                    cweno3(a1, a2, a3, &xl, &xr);
                    uR[k] = xl;
                    cL[k] = a1; cR[k] = a2;
                }
                if (!Q) {
                    maxwellian_e3(uL, qL);
                    maxwellian_e3(uR, qR);
                }
                for (int k = 0; Q && k < nq; ++k) {
                    int ox = dir == 0, oy = dir == 1;
                    double a0 = fetch(c, Q, nq, k, lx - ox, ly - oy, 1);
                    double a1 = fetch(c, Q, nq, k, lx, ly, 1);
                    double a2 = fetch(c, Q, nq, k, rx, ry, 1);
                    double a3 = fetch(c, Q, nq, k, rx + ox, ry + oy, 1);
                    double xl, xr;
                    cweno3(a0, a1, a2, &xl, &xr);
                    qL[k] = xr;
                    cweno3(a1, a2, a3, &xl, &xr);
                    qR[k] = xl;
                }
                double a = wave_speed(d, dir, cL);
                double ar = wave_speed(d, dir, cR);
                if (ar > a) a = ar;
                double H[10];
                for (int k = 0; k < nc; ++k)
                    H[k] = 0.5 * (flux_comp(d, dir, k, uL, qL) + flux_comp(d, dir, k, uR, qR)) -
                           0.5 * a * (uR[k] - uL[k]);
                long li = (long)ly * g->nx + lx;
                for (int k = 0; k < nc; ++k) out[li * nc + k] -= H[k] / h;
                /* right cell (skip the wall: no cell beyond it) */
                int rxx = ((rx % g->nx) + g->nx) % g->nx, ryy = ry;
                if (ryy >= g->ny) {
                    if (g->bc_y == 1) continue;
                    ryy = 0;
                }
                long ri = (long)ryy * g->nx + rxx;
                for (int k = 0; k < nc; ++k) out[ri * nc + k] += H[k] / h;
            }
        /* bottom wall interface (y = y0) for walls: flux into cell row 0 */
        if (dir == 1 && g->bc_y == 1) {
            for (int ix = 0; ix < g->nx; ++ix) {
                double uL[10], uR[10], qL[10], qR[10], cL[10], cR[10];
                for (int k = 0; k < nc; ++k) {
                    double a0 = fetch(c, U, nc, k, ix, -2, 0);
                    double a1 = fetch(c, U, nc, k, ix, -1, 0);
                    double a2 = fetch(c, U, nc, k, ix, 0, 0);
                    double a3 = fetch(c, U, nc, k, ix, 1, 0);
                    double xl, xr;
                    cweno3(a0, a1, a2, &xl, &xr);
                    uL[k] = xr;
                    cweno3(a1, a2, a3, &xl, &xr);
                    uR[k] = xl;
                    cL[k] = a1; cR[k] = a2;
                }
                if (!Q) {
                    maxwellian_e3(uL, qL);
                    maxwellian_e3(uR, qR);
                }
                for (int k = 0; Q && k < nq; ++k) {
                    double a0 = fetch(c, Q, nq, k, ix, -2, 1);
                    double a1 = fetch(c, Q, nq, k, ix, -1, 1);
                    double a2 = fetch(c, Q, nq, k, ix, 0, 1);
                    double a3 = fetch(c, Q, nq, k, ix, 1, 1);
                    double xl, xr;
                    cweno3(a0, a1, a2, &xl, &xr);
                    qL[k] = xr;
                    cweno3(a1, a2, a3, &xl, &xr);
                    qR[k] = xl;
                }
                double a = wave_speed(d, 1, cL), ar = wave_speed(d, 1, cR);
                if (ar > a) a = ar;
                for (int k = 0; k < nc; ++k) {
                    double H = 0.5 * (flux_comp(d, 1, k, uL, qL) + flux_comp(d, 1, k, uR, qR)) -
                               0.5 * a * (uR[k] - uL[k]);
                    out[(long)ix * nc + k] += H / g->dy;
                }
            }
        }
    }
    /* Lorentz sources */
    for (long i = 0; i < ncell; ++i) {
        const double* u = U + i * nc;
        const double* eb = EB + i * 6;
        double* o = out + i * nc;
        if (d == 1) {
            o[1] += qm * u[0] * eb[0];
            o[2] += qm * 2.0 * u[1] * eb[0];
            continue;
        }
        const double* E = eb;
        const double* B = eb + 3;
        const double* nu = u + 1;
        o[1] += qm * (u[0] * E[0] + nu[1] * B[2] - nu[2] * B[1]);
        o[2] += qm * (u[0] * E[1] + nu[2] * B[0] - nu[0] * B[2]);
        o[3] += qm * (u[0] * E[2] + nu[0] * B[1] - nu[1] * B[0]);
        double E2m[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) E2m[a][b] = u[4 + sym2(a, b)];
        double C[3][3];
        for (int a = 0; a < 3; ++a) {
            /* (row a of E2) x B */
            C[a][0] = E2m[a][1] * B[2] - E2m[a][2] * B[1];
            C[a][1] = E2m[a][2] * B[0] - E2m[a][0] * B[2];
            C[a][2] = E2m[a][0] * B[1] - E2m[a][1] * B[0];
        }
        for (int a = 0; a < 3; ++a)
            for (int b = a; b < 3; ++b)
                o[4 + sym2(a, b)] += qm * (nu[a] * E[b] + nu[b] * E[a] + C[a][b] + C[b][a]);
    }
}

int or_fluid_step(double* U, const or_grid* g, const or_species* sp,
                  const double* Q0, const double* Qh, const double* Q1,
                  const double* EB, double dt) {
    fl_ctx c;
    c.g = g; c.sp = sp;
    c.ncomp = g->nvdim == 1 ? 3 : 10;
    c.nq = g->nvdim == 1 ? 1 : 10;
    long n = (long)g->nx * g->ny * c.ncomp;
    double* L = (double*)malloc(sizeof(double) * (size_t)n);
    double* U1 = (double*)malloc(sizeof(double) * (size_t)n);
    double* U2 = (double*)malloc(sizeof(double) * (size_t)n);
    rhs(&c, U, Q0, EB, L);
    for (long i = 0; i < n; ++i) U1[i] = U[i] + dt * L[i];
    rhs(&c, U1, Q1, EB, L);
    for (long i = 0; i < n; ++i) U2[i] = 0.75 * U[i] + 0.25 * (U1[i] + dt * L[i]);
    rhs(&c, U2, Qh, EB, L);
    for (long i = 0; i < n; ++i) U[i] = U[i] / 3.0 + 2.0 / 3.0 * (U2[i] + dt * L[i]);
    free(L); free(U1); free(U2);
    return 0;
}

/* The heat-flux closure of Sec. 2.3, Eq. (gradient closure):
 *   div Q_s = -(chi / k_s0) n_s v_ts lap T_s,  chi = 2 sqrt(2/pi),
 *   v_ts = sqrt(tr(T_s) / (3 m_s)), k_s0 = 1/d_s,
 * so the second-moment equation (divided by m, T = m theta) gains the source
 * -(1/m) div Q = (chi / k_s0) n v_t lap theta, with the five-point Laplacian
 * of theta at cell centres (ghost cells as for the state: periodic, or the
 * mirror cell with the parity of the component beyond a wall). */
static void closure_source(const fl_ctx* c, const double* U, double chi_k0, double* out) {
    const or_grid* g = c->g;
    for (int iy = 0; iy < g->ny; ++iy)
        for (int ix = 0; ix < g->nx; ++ix) {
            double t0[6], txm[6], txp[6], tym[6], typ[6];
            theta_at(c, U, ix, iy, t0);
            theta_at(c, U, ix - 1, iy, txm);
            theta_at(c, U, ix + 1, iy, txp);
            theta_at(c, U, ix, iy - 1, tym);
            theta_at(c, U, ix, iy + 1, typ);
            long i = (long)iy * g->nx + ix;
            double n = U[i * 10];
            double tr = t0[0] + t0[3] + t0[5];
            double vt = sqrt(tr > 0.0 ? tr / 3.0 : 0.0);
            for (int k = 0; k < 6; ++k) {
                double lap = (txp[k] - 2.0 * t0[k] + txm[k]) / (g->dx * g->dx) +
                             (typ[k] - 2.0 * t0[k] + tym[k]) / (g->dy * g->dy);
                out[i * 10 + 4 + k] += chi_k0 * n * vt * lap;
            }
        }
}

int or_fluid_step_closure(double* U, const or_grid* g, const or_species* sp,
                          const double* EB, double dt, double chi_k0) {
    if (g->nvdim != 3) return -1;
    fl_ctx c;
    c.g = g; c.sp = sp;
    c.ncomp = 10;
    c.nq = 10;
    long n = (long)g->nx * g->ny * c.ncomp;
    double* L = (double*)malloc(sizeof(double) * (size_t)n);
    double* U1 = (double*)malloc(sizeof(double) * (size_t)n);
    double* U2 = (double*)malloc(sizeof(double) * (size_t)n);
    rhs(&c, U, NULL, EB, L);
    closure_source(&c, U, chi_k0, L);
    for (long i = 0; i < n; ++i) U1[i] = U[i] + dt * L[i];
    rhs(&c, U1, NULL, EB, L);
    closure_source(&c, U1, chi_k0, L);
    for (long i = 0; i < n; ++i) U2[i] = 0.75 * U[i] + 0.25 * (U1[i] + dt * L[i]);
    rhs(&c, U2, NULL, EB, L);
    closure_source(&c, U2, chi_k0, L);
    for (long i = 0; i < n; ++i) U[i] = U[i] / 3.0 + 2.0 / 3.0 * (U2[i] + dt * L[i]);
    free(L); free(U1); free(U2);
    return 0;
}

int or_fluid_rhs_closure(const double* U, const or_grid* g, const or_species* sp,
                         const double* EB, double chi_k0, double* out) {
    if (g->nvdim != 3) return -1;
    fl_ctx c;
    c.g = g; c.sp = sp;
    c.ncomp = 10;
    c.nq = 10;
    rhs(&c, U, NULL, EB, out);
    closure_source(&c, U, chi_k0, out);
    return 0;
}

void or_maxwellian_e3(const double* u, double* e3) { maxwellian_e3(u, e3); }
