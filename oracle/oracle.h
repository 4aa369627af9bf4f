/*
 * Plain FP64 CPU oracle of the moment-fitting PFC Vlasov solver
 * (Allmann-Rahn, Lautenbach, Grauer, arXiv:2109.06743).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library. It shares no code
 * with the CUDA path and is written for clarity, not speed: every routine
 * follows the paper's definitions step by step with plain loops.
 *
 * Layout (same logical layout as the GPU path, but its own definitions):
 *   f[y][x][vz][vy][vx]   (2D3V)   or   f[x][v]  (1D1V, ny = 1)
 * Velocity cell centres: v_a(i) = vmin_a + (i + 1/2) dv_a.
 * Raw moments per spatial cell ("M" below): midpoint sums
 *   M_alpha = dv^3 * sum_c v_c^alpha f_c,
 * ordered 1, x, y, z, xx, xy, xz, yy, yz, zz, xxx, xxy, xxz, xyy, xyz, xzz,
 * yyy, yyz, yzz, zzz (20 values; 1D1V: 1, v, vv, vvv = 4 values).
 */
#ifndef VLASOV_ORACLE_H
#define VLASOV_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nvdim;          /* velocity dimensions: 1 (1D1V) or 3 (2D3V)       */
    int nx, ny;         /* spatial cells (ny = 1 for 1D1V)                 */
    double x0, dx;      /* left edge and width of spatial cells in x       */
    double y0, dy;      /* same in y                                       */
    int bc_y;           /* 0: periodic in y, 1: reflecting/conducting walls */
} or_grid;

typedef struct {
    double q, m;        /* charge and mass (normalised units)              */
    int nv[3];          /* velocity cells per axis (1D1V: nv[1]=nv[2]=1)   */
    double vmin[3];     /* lower edge of the velocity box                  */
    double dv[3];       /* velocity cell widths                            */
} or_species;

/* ---- PFC scheme (Filbet, Sonnendruecker, Bertrand 2001; paper Sec. 2.1) -- */
/* One conservative 1D step of the PFC scheme on an extended line.
 * fext holds n cells plus ng ghost cells on each side (cell i at fext[ng+i]).
 * c is the displacement in cell widths (a*dt/dx). zero_flux forces the two
 * boundary-interface fluxes to zero. Returns 0, or -1 if ng < floor(|c|)+2. */
int or_pfc_line(const double* fext, int n, int ng, double c, int zero_flux,
                double* out);

/* Spatial sweep of species s along axis 0 (x, periodic) or 1 (y, periodic or
 * reflecting walls: ghosts f(-y, v_y) = f(y, -v_y)). In place. */
int or_advect_space(double* f, const or_grid* g, const or_species* sp,
                    int axis, double dt);

/* Velocity-space advection under (q/m)(E + v x B) over dt at every spatial
 * cell. EB is cell centred, [ncell][6] = Ex Ey Ez Bx By Bz. nshear = 5 uses
 * the exact shear factorisation of the Boris map, 3 the plain x,y,z split.
 * Zero-flux boundaries at the velocity box. In place.
 * Pinned: the five shears compose to the Boris map, rest invariance, E x B
 * drift. Parity unpinned: agreement with the paper's own velocity splitting
 * (its backsubstitution sweeps are cited, not given). */
int or_advect_velocity(double* f, const or_grid* g, const or_species* sp,
                       const double* EB, double dt, int nshear);

/* Shear factors of the velocity map of one cell: for sweep k (k < nshear),
 * out[k*4+0] = axis, out[k*4+1], out[k*4+2] = coefficients of the two other
 * velocity components (in increasing axis order), out[k*4+3] = constant.
 * The sweep moves v_axis by coef1*v_b + coef2*v_c + const. */
int or_velocity_shears(double qm, const double* E, const double* B, double dt,
                       int nshear, double* out);

/* ---- Moments (paper Sec. 2.1) ------------------------------------------- */
void or_moments(const double* f, const or_grid* g, const or_species* sp,
                double* out);

/* ---- Discrete ten-moment Maxwellian fit and exchange (Sec. 2.2) --------- */
/* Fit theta = (n', u', Theta') so that the midpoint moments of degree <= 2 of
 * the sampled Maxwellian equal target = (n, nu, int v v f) (10 values, or 3
 * for 1D1V). Newton iteration. status: 0 converged, 1 fallback to the
 * continuous Maxwellian of the targets, 2 invalid targets (theta n' = 0). */
int or_maxent_fit(const double* target, const or_species* sp, int nvdim,
                  double tol, int max_iter, double* theta, int* iters,
                  int* status);

/* Sample the ten-moment Maxwellian with parameters theta on the grid. */
void or_maxwellian_grid(const double* theta, const or_species* sp, int nvdim,
                        double* out);

/* Moment fitting of Algorithm 1 for one species: V targets from f, F targets
 * from the fluid state (rescaled by n_V/n_F), two fits, exchange
 * f <- f - f_M,V + f_M,F, limiter (clip negatives, rescale to n_V). The fluid
 * state is replaced by its rescaled moments. stats[0] += Newton iterations,
 * stats[1] += fallbacks, stats[2] += clipped cells. */
int or_moment_fit(double* f, const or_grid* g, const or_species* sp,
                  double* fluid, double tol, int max_iter, long* stats);

/* ---- Ten-moment fluid (Sec. 2.1 eqs.; CWENO + SSP-RK3) ------------------ */
/* U[ncell][ncomp] with ncomp = 10 (n, nu_a, E2_ab) or 3 (n, nu, E2) per
 * species, E2 = P/m = int v v f. Q0, Qh, Q1: third moments int v v v f at t,
 * t+dt/2 and t+dt, [ncell][10] (1D1V: [ncell][1]). EB frozen, cell centred. */
int or_fluid_step(double* U, const or_grid* g, const or_species* sp,
                  const double* Q0, const double* Qh, const double* Q1,
                  const double* EB, double dt);
/* The stand-alone fluid model with the gradient heat-flux closure (Sec. 2.3):
 * the third moment in the flux is that of the state's Maxwellian, and the
 * heat flux enters as chi_k0 n v_t lap(theta) in the second-moment equation
 * (chi_k0 = chi / k_s0). 2D3V only. One SSP-RK3 step with EB frozen; the
 * right-hand side alone (out[ncell][10]) for tests. */
int or_fluid_step_closure(double* U, const or_grid* g, const or_species* sp,
                          const double* EB, double dt, double chi_k0);
int or_fluid_rhs_closure(const double* U, const or_grid* g, const or_species* sp,
                         const double* EB, double chi_k0, double* out);
/* E3 of the closure model for one state (n, nu_a, E2_ab) -> [10] */
void or_maxwellian_e3(const double* u, double* e3);

/* ---- Fields ------------------------------------------------------------- */
/* Yee fields, one array of 6 planes, each [ny+1][nx]:
 * Ex(i+1/2, j), Ey(i, j+1/2), Ez(i, j), Bx(i, j+1/2), By(i+1/2, j),
 * Bz(i+1/2, j+1/2) with i, j integer cell corners and cell (i, j) spanning
 * [x_i, x_{i+1}] x [y_j, y_{j+1}]. Planes with a j+1/2 position use rows
 * 0..ny-1. One leapfrog FDTD step of length h with the cell-centred current
 * J[ncell][3]; c is the speed of light (mu0 = 1, eps0 = 1/c^2). */
int or_maxwell(double* yee, const or_grid* g, const double* J, double h,
               double c);
/* Average Yee fields to cell centres: EB[ncell][6]. */
void or_fields_to_centres(const double* yee, const or_grid* g, double* EB);
/* 1D periodic Poisson dE/dx = rho (eps0 = 1): E at cell centres, zero mean. */
void or_poisson_1d(const double* rho, int nx, double dx, double* E);

#ifdef __cplusplus
}
#endif
#endif
