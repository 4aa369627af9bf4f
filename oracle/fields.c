/*
 * Oracle: field solvers (test infrastructure only; see oracle.h).
 *
 * Paper Sec. 2.1: Maxwell's equations solved by the FDTD (Yee) method, split
 * into two half steps per time step (Algorithm 1); mu0 = 1 and eps0 = 1/c^2
 * in the electromagnetic normalisation. Sec. 3.3: conducting walls for the
 * fields in y. Sec. 3.1: a Poisson solver for the electrostatic runs
 * (eps0 = 1, dE/dx = rho).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

enum { EX = 0, EY = 1, EZ = 2, BX = 3, BY = 4, BZ = 5 };

typedef struct {
    int nx, ny, wall;
    long plane;
} yee_t;

static double* P(double* yee, const yee_t* y, int comp) { return yee + comp * y->plane; }

static long at(const yee_t* y, int i, int j) {
    i = ((i % y->nx) + y->nx) % y->nx;
    return (long)j * y->nx + i;
}

/* row j of a j+1/2 plane, with periodic wrap in y when there are no walls */
static int wrap_half(const yee_t* y, int j) {
    if (y->wall) return j;
    return ((j % y->ny) + y->ny) % y->ny;
}
/* row j of an integer-j plane (0..ny); periodic: row ny duplicates row 0 */
static int wrap_int(const yee_t* y, int j) {
    if (y->wall) return j;
    return ((j % y->ny) + y->ny) % y->ny;
}

static void faraday(double* yee, const yee_t* y, double h, double dx, double dy) {
    double *Ex = P(yee, y, EX), *Ey = P(yee, y, EY), *Ez = P(yee, y, EZ);
    double *Bx = P(yee, y, BX), *By = P(yee, y, BY), *Bz = P(yee, y, BZ);
    /* Bx(i, j+1/2) -= h dEz/dy */
    for (int j = 0; j < y->ny; ++j)
        for (int i = 0; i < y->nx; ++i)
            Bx[at(y, i, j)] -= h * (Ez[at(y, i, wrap_int(y, j + 1))] - Ez[at(y, i, j)]) / dy;
    /* By(i+1/2, j) += h dEz/dx  (rows 0..ny; walls keep Ez = 0) */
    int jmax = y->wall ? y->ny : y->ny - 1;
    for (int j = 0; j <= jmax; ++j)
        for (int i = 0; i < y->nx; ++i)
            By[at(y, i, j)] += h * (Ez[at(y, i + 1, j)] - Ez[at(y, i, j)]) / dx;
    /* Bz(i+1/2, j+1/2) -= h (dEy/dx - dEx/dy) */
    for (int j = 0; j < y->ny; ++j)
        for (int i = 0; i < y->nx; ++i)
            Bz[at(y, i, j)] -= h * ((Ey[at(y, i + 1, j)] - Ey[at(y, i, j)]) / dx -
                                    (Ex[at(y, i, wrap_int(y, j + 1))] - Ex[at(y, i, j)]) / dy);
    if (!y->wall)
        for (int i = 0; i < y->nx; ++i) By[at(y, i, y->ny)] = By[at(y, i, 0)];
}

/* cell-centred current J[cell][3] at the Yee positions */
static double jx_at(const double* J, const yee_t* y, int i, int j) {
    /* Ex point (i+1/2, j): average of cells (i, j-1) and (i, j) */
    int ja = wrap_half(y, j - 1), jb = wrap_half(y, j);
    return 0.5 * (J[at(y, i, ja) * 3 + 0] + J[at(y, i, jb) * 3 + 0]);
}
static double jy_at(const double* J, const yee_t* y, int i, int j) {
    return 0.5 * (J[at(y, i - 1, j) * 3 + 1] + J[at(y, i, j) * 3 + 1]);
}
static double jz_at(const double* J, const yee_t* y, int i, int j) {
    int ja = wrap_half(y, j - 1), jb = wrap_half(y, j);
    return 0.25 * (J[at(y, i - 1, ja) * 3 + 2] + J[at(y, i, ja) * 3 + 2] +
                   J[at(y, i - 1, jb) * 3 + 2] + J[at(y, i, jb) * 3 + 2]);
}

static void ampere(double* yee, const yee_t* y, const double* J, double h,
                   double c2, double dx, double dy) {
    double *Ex = P(yee, y, EX), *Ey = P(yee, y, EY), *Ez = P(yee, y, EZ);
    double *Bx = P(yee, y, BX), *By = P(yee, y, BY), *Bz = P(yee, y, BZ);
    int j0 = y->wall ? 1 : 0, j1 = y->wall ? y->ny - 1 : y->ny - 1;
    /* Ex(i+1/2, j) += h c^2 (dBz/dy - Jx), interior rows (walls: Ex = 0) */
    for (int j = j0; j <= j1; ++j)
        for (int i = 0; i < y->nx; ++i)
            Ex[at(y, i, j)] += h * c2 * ((Bz[at(y, i, j)] - Bz[at(y, i, wrap_half(y, j - 1))]) / dy -
                                         jx_at(J, y, i, j));
    /* Ey(i, j+1/2) += h c^2 (-dBz/dx - Jy) */
    for (int j = 0; j < y->ny; ++j)
        for (int i = 0; i < y->nx; ++i)
            Ey[at(y, i, j)] += h * c2 * (-(Bz[at(y, i, j)] - Bz[at(y, i - 1, j)]) / dx -
                                         jy_at(J, y, i, j));
    /* Ez(i, j) += h c^2 (dBy/dx - dBx/dy - Jz) */
    for (int j = j0; j <= j1; ++j)
        for (int i = 0; i < y->nx; ++i)
            Ez[at(y, i, j)] += h * c2 * ((By[at(y, i, j)] - By[at(y, i - 1, j)]) / dx -
                                         (Bx[at(y, i, j)] - Bx[at(y, i, wrap_half(y, j - 1))]) / dy -
                                         jz_at(J, y, i, j));
    if (y->wall) {
        for (int i = 0; i < y->nx; ++i) {
            Ex[at(y, i, 0)] = 0.0; Ex[at(y, i, y->ny)] = 0.0;
            Ez[at(y, i, 0)] = 0.0; Ez[at(y, i, y->ny)] = 0.0;
        }
    } else {
        for (int i = 0; i < y->nx; ++i) {
            Ex[at(y, i, y->ny)] = Ex[at(y, i, 0)];
            Ez[at(y, i, y->ny)] = Ez[at(y, i, 0)];
        }
    }
}

int or_maxwell(double* yee, const or_grid* g, const double* J, double h,
               double c) {
    if (g->nvdim != 3) return -1;
    yee_t y = {g->nx, g->ny, g->bc_y == 1, (long)(g->ny + 1) * g->nx};
    faraday(yee, &y, 0.5 * h, g->dx, g->dy);
    ampere(yee, &y, J, h, c * c, g->dx, g->dy);
    faraday(yee, &y, 0.5 * h, g->dx, g->dy);
    return 0;
}

void or_fields_to_centres(const double* yee, const or_grid* g, double* EB) {
    yee_t y = {g->nx, g->ny, g->bc_y == 1, (long)(g->ny + 1) * g->nx};
    const double* Ex = yee + EX * y.plane;
    const double* Ey = yee + EY * y.plane;
    const double* Ez = yee + EZ * y.plane;
    const double* Bx = yee + BX * y.plane;
    const double* By = yee + BY * y.plane;
    const double* Bz = yee + BZ * y.plane;
    for (int j = 0; j < g->ny; ++j)
        for (int i = 0; i < g->nx; ++i) {
            double* o = EB + ((long)j * g->nx + i) * 6;
            o[0] = 0.5 * (Ex[at(&y, i, j)] + Ex[at(&y, i, j + 1)]);
            o[1] = 0.5 * (Ey[at(&y, i, j)] + Ey[at(&y, i + 1, j)]);
            o[2] = 0.25 * (Ez[at(&y, i, j)] + Ez[at(&y, i + 1, j)] + Ez[at(&y, i, j + 1)] +
                           Ez[at(&y, i + 1, j + 1)]);
            o[3] = 0.5 * (Bx[at(&y, i, j)] + Bx[at(&y, i + 1, j)]);
            o[4] = 0.5 * (By[at(&y, i, j)] + By[at(&y, i, j + 1)]);
            o[5] = Bz[at(&y, i, j)];
        }
}

void or_poisson_1d(const double* rho, int nx, double dx, double* E) {
    /* face values E_{i+1/2} = E_{i-1/2} + dx rho_i, then zero mean */
    double* Ef = (double*)malloc(sizeof(double) * (size_t)nx);
    double acc = 0.0;
    for (int i = 0; i < nx; ++i) {
        acc += dx * rho[i];
        Ef[i] = acc; /* E at face i + 1/2, up to a constant */
    }
    double mean = 0.0;
    for (int i = 0; i < nx; ++i) mean += Ef[i];
    mean /= nx;
    for (int i = 0; i < nx; ++i) Ef[i] -= mean;
    for (int i = 0; i < nx; ++i) {
        double left = Ef[(i - 1 + nx) % nx];
        E[i] = 0.5 * (left + Ef[i]);
    }
    free(Ef);
}
