/*
 * Oracle: velocity moments (test infrastructure only; see oracle.h).
 *
 * Paper Sec. 2.1: n = int f dv, u = (1/n) int v f dv, P = m int v v f dv,
 * Q = m int v v v f dv. The integrals are taken with the midpoint rule at the
 * velocity cell centres (the paper does not say how it integrates; this is
 * the reading used throughout). The mass factor m is left out: the oracle
 * returns the raw sums int v^alpha f dv, alpha of degree 0..3.
 */
#include "oracle.h"

static const int MONO3[20][3] = {
    {0, 0, 0},
    {1, 0, 0}, {0, 1, 0}, {0, 0, 1},
    {2, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2},
    {3, 0, 0}, {2, 1, 0}, {2, 0, 1}, {1, 2, 0}, {1, 1, 1}, {1, 0, 2},
    {0, 3, 0}, {0, 2, 1}, {0, 1, 2}, {0, 0, 3},
};

static double ipow(double x, int p) {
    double r = 1.0;
    for (int k = 0; k < p; ++k) r *= x;
    return r;
}

void or_moments(const double* f, const or_grid* g, const or_species* sp,
                double* out) {
    long ncell = (long)g->nx * g->ny;
    if (g->nvdim == 1) {
        int n = sp->nv[0];
        for (long c = 0; c < ncell; ++c) {
            double m[4] = {0.0, 0.0, 0.0, 0.0};
            for (int i = 0; i < n; ++i) {
                double v = sp->vmin[0] + (i + 0.5) * sp->dv[0];
                double fv = f[c * n + i];
                for (int p = 0; p < 4; ++p) m[p] += ipow(v, p) * fv;
            }
            for (int p = 0; p < 4; ++p) out[c * 4 + p] = m[p] * sp->dv[0];
        }
        return;
    }
    int nx = sp->nv[0], ny = sp->nv[1], nz = sp->nv[2];
    long V = (long)nx * ny * nz;
    double dv3 = sp->dv[0] * sp->dv[1] * sp->dv[2];
    for (long c = 0; c < ncell; ++c) {
        double m[20];
        for (int a = 0; a < 20; ++a) m[a] = 0.0;
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    double v[3] = {sp->vmin[0] + (i + 0.5) * sp->dv[0],
                                   sp->vmin[1] + (j + 0.5) * sp->dv[1],
                                   sp->vmin[2] + (k + 0.5) * sp->dv[2]};
                    double fv = f[c * V + ((long)k * ny + j) * nx + i];
                    for (int a = 0; a < 20; ++a)
                        m[a] += ipow(v[0], MONO3[a][0]) * ipow(v[1], MONO3[a][1]) *
                                ipow(v[2], MONO3[a][2]) * fv;
                }
        for (int a = 0; a < 20; ++a) out[c * 20 + a] = m[a] * dv3;
    }
}
