/*
 * Oracle: PFC advection (test infrastructure only; see oracle.h).
 *
 * The paper advances f with the third-order positive flux-conservative (PFC)
 * scheme of Filbet, Sonnendruecker and Bertrand (2001), cited in Sec. 1 and
 * Sec. 2.1, with zero-flux boundaries in velocity space (Sec. 2.1) and
 * reflecting walls in y for the GEM setup (Sec. 3.3). The velocity-space
 * splitting is the "backsubstitution" of Schmitz and Grauer (2006b), whose
 * details the paper does not give; the reading used here is an exact
 * factorisation of the Boris map into five single-axis shears.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- PFC --- */

/* Positivity limiters of the PFC reconstruction in cell j (Filbet et al.,
 * with the upper bound f_infinity taken as +infinity: positivity only). */
static double eps_plus(double fjm1, double fj, double fjp1) {
    (void)fjm1;
    double d = fjp1 - fj;
    if (d > 0.0) {
        double r = 2.0 * fj / d;
        return r < 1.0 ? r : 1.0;
    }
    return 1.0;
}

static double eps_minus(double fjm1, double fj, double fjp1) {
    (void)fjp1;
    double d = fj - fjm1;
    if (d < 0.0) {
        double r = -2.0 * fj / d;
        return r < 1.0 ? r : 1.0;
    }
    return 1.0;
}

/* Integral over the part of cell j that crosses the downstream interface
 * during dt, in units of f * dx, for a positive displacement with fractional
 * part alpha: the limited cubic reconstruction of the primitive. */
static double flux_frac_pos(double alpha, double fjm1, double fj, double fjp1) {
    double ep = eps_plus(fjm1, fj, fjp1), em = eps_minus(fjm1, fj, fjp1);
    return alpha * (fj + ep * (1.0 - alpha) * (2.0 - alpha) / 6.0 * (fjp1 - fj)
                       + em * (1.0 - alpha) * (1.0 + alpha) / 6.0 * (fj - fjm1));
}

/* Mirror image for a negative displacement: the part of cell j that leaves
 * through its left interface. */
static double flux_frac_neg(double alpha, double fjm1, double fj, double fjp1) {
    double ep = eps_plus(fjm1, fj, fjp1), em = eps_minus(fjm1, fj, fjp1);
    return alpha * (fj - ep * (1.0 - alpha) * (1.0 + alpha) / 6.0 * (fjp1 - fj)
                       - em * (1.0 - alpha) * (2.0 - alpha) / 6.0 * (fj - fjm1));
}

int or_pfc_line(const double* fext, int n, int ng, double c, int zero_flux,
                double* out) {
    double a = fabs(c);
    int s = (int)floor(a);
    double alpha = a - s;
    if (ng < s + 2) return -1;
    const double* f = fext + ng; /* f[i], valid for -ng <= i < n + ng */
    /* Phi[k] is the flux (in cell units) through interface k - 1/2, k=0..n */
    double* Phi = (double*)malloc(sizeof(double) * (size_t)(n + 1));
    for (int k = 0; k <= n; ++k) {
        int i = k - 1; /* interface i + 1/2 */
        double phi;
        if (c >= 0.0) {
            int j = i - s; /* cell holding the foot of the characteristic */
            double sum = 0.0;
            for (int m = j + 1; m <= i; ++m) sum += f[m];
            phi = sum + flux_frac_pos(alpha, f[j - 1], f[j], f[j + 1]);
        } else {
            int j = i + 1 + s;
            double sum = 0.0;
            for (int m = i + 1; m <= i + s; ++m) sum += f[m];
            phi = -(sum + flux_frac_neg(alpha, f[j - 1], f[j], f[j + 1]));
        }
        Phi[k] = phi;
    }
    if (zero_flux) {
        Phi[0] = 0.0;
        Phi[n] = 0.0;
    }
    for (int i = 0; i < n; ++i) out[i] = f[i] + Phi[i] - Phi[i + 1];
    free(Phi);
    return 0;
}

/* ------------------------------------------------------- spatial sweeps --- */

static long vblock(const or_grid* g, const or_species* sp) {
    return g->nvdim == 1 ? sp->nv[0] : (long)sp->nv[0] * sp->nv[1] * sp->nv[2];
}

static double vcentre(const or_species* sp, int axis, int idx) {
    return sp->vmin[axis] + (idx + 0.5) * sp->dv[axis];
}

int or_advect_space(double* f, const or_grid* g, const or_species* sp,
                    int axis, double dt) {
    if (axis != 0 && axis != 1) return -1;
    if (axis == 1 && g->nvdim != 3) return -1;
    long V = vblock(g, sp);
    long ncell = (long)g->nx * g->ny;
    int n = axis == 0 ? g->nx : g->ny;
    double h = axis == 0 ? g->dx : g->dy;
    int wall = (axis == 1 && g->bc_y == 1);
    int nvx = sp->nv[0], nvy = g->nvdim == 3 ? sp->nv[1] : 1;

    double* old = (double*)malloc(sizeof(double) * (size_t)(ncell * V));
    memcpy(old, f, sizeof(double) * (size_t)(ncell * V));

    double vmax_abs = 0.0;
    for (int i = 0; i < sp->nv[axis]; ++i) {
        double v = fabs(vcentre(sp, axis, i));
        if (v > vmax_abs) vmax_abs = v;
    }
    int ng = (int)floor(vmax_abs * fabs(dt) / h) + 3;
    if (wall && ng > n) { free(old); return -3; }
    double* ext = (double*)malloc(sizeof(double) * (size_t)(n + 2 * ng));
    double* res = (double*)malloc(sizeof(double) * (size_t)n);

    int other = axis == 0 ? g->ny : g->nx;
    for (int o = 0; o < other; ++o) {
        for (long vi = 0; vi < V; ++vi) {
            int ivx = (int)(vi % nvx);
            int ivy = (int)((vi / nvx) % nvy);
            int iva = axis == 0 ? ivx : ivy;
            double c = vcentre(sp, axis, iva) * dt / h;
            /* mirrored velocity index (v_y -> -v_y) for wall ghosts */
            long vmir = vi + (long)(nvy - 1 - 2 * ivy) * nvx;
            for (int k = -ng; k < n + ng; ++k) {
                int cell = k;
                long vsrc = vi;
                if (k < 0 || k >= n) {
                    if (wall) {
                        cell = k < 0 ? -1 - k : 2 * n - 1 - k;
                        vsrc = vmir;
                    } else {
                        cell = ((k % n) + n) % n;
                    }
                }
                long sidx = axis == 0 ? ((long)o * g->nx + cell) : ((long)cell * g->nx + o);
                ext[k + ng] = old[sidx * V + vsrc];
            }
            if (or_pfc_line(ext, n, ng, c, 0, res) != 0) {
                free(old); free(ext); free(res);
                return -2;
            }
            for (int k = 0; k < n; ++k) {
                long sidx = axis == 0 ? ((long)o * g->nx + k) : ((long)k * g->nx + o);
                f[sidx * V + vi] = res[k];
            }
        }
    }
    free(old); free(ext); free(res);
    return 0;
}

/* ------------------------------------------------------ velocity sweeps --- */

static void cross(const double* a, const double* b, double* out) {
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

/* Boris rotation of w (no electric kick): w' = w + w x t, w+ = w + w' x s,
 * t = (q/m) B dt / 2, s = 2 t / (1 + t.t). */
static void boris_rotate(const double* w, const double* t, const double* s,
                         double* out) {
    double wp[3], c1[3], c2[3];
    cross(w, t, c1);
    for (int a = 0; a < 3; ++a) wp[a] = w[a] + c1[a];
    cross(wp, s, c2);
    for (int a = 0; a < 3; ++a) out[a] = w[a] + c2[a];
}

/* Row operation on matrix M (3x3 row-major): row r += c1*row(o1) + c2*row(o2) */
static void row_op(double M[3][3], int r, int o1, double c1, int o2, double c2) {
    for (int col = 0; col < 3; ++col) M[r][col] += c1 * M[o1][col] + c2 * M[o2][col];
}

static void others(int axis, int* b, int* c) {
    if (axis == 0) { *b = 1; *c = 2; }
    else if (axis == 1) { *b = 0; *c = 2; }
    else { *b = 0; *c = 1; }
}

int or_velocity_shears(double qm, const double* E, const double* B, double dt,
                       int nshear, double* out) {
    if (nshear == 3) {
        /* plain split: each 1D sweep uses the Lorentz acceleration with the
         * other two components at their (already updated) grid values */
        for (int k = 0; k < 3; ++k) {
            int b, c;
            others(k, &b, &c);
            /* (v x B)_k = v_{k+1} B_{k+2} - v_{k+2} B_{k+1} (cyclic) */
            double cb = 0.0, cc = 0.0;
            int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
            /* coefficient of v_k1 is B_k2, of v_k2 is -B_k1 */
            if (b == k1) { cb = B[k2]; cc = -B[k1]; }
            else { cb = -B[k1]; cc = B[k2]; }
            out[k * 4 + 0] = k;
            out[k * 4 + 1] = qm * dt * cb;
            out[k * 4 + 2] = qm * dt * cc;
            out[k * 4 + 3] = qm * dt * E[k];
        }
        return 0;
    }
    if (nshear != 5) return -1;

    /* The Boris map V = R (v + h) + h with h = (q/m) E dt / 2. D = R - I is
     * formed directly, (R - I) w = (w + w x t) x s, so that the diagonal
     * deviations carry no cancellation. */
    double t[3], s[3], tt = 0.0;
    for (int a = 0; a < 3; ++a) { t[a] = 0.5 * qm * dt * B[a]; tt += t[a] * t[a]; }
    for (int a = 0; a < 3; ++a) s[a] = 2.0 * t[a] / (1.0 + tt);
    double D[3][3];
    for (int col = 0; col < 3; ++col) {
        double e[3] = {0.0, 0.0, 0.0}, wt[3], w1[3], r[3];
        e[col] = 1.0;
        cross(e, t, wt);
        for (int a = 0; a < 3; ++a) w1[a] = e[a] + wt[a];
        cross(w1, s, r);
        for (int row = 0; row < 3; ++row) D[row][col] = r[row];
    }
    double h[3], bvec[3];
    for (int a = 0; a < 3; ++a) h[a] = 0.5 * qm * dt * E[a];
    for (int a = 0; a < 3; ++a) bvec[a] = D[a][0] * h[0] + D[a][1] * h[1] + D[a][2] * h[2] + 2.0 * h[a];

    /* Pivot: the axis with the largest |B| component plays the role of the
     * first (and last) sweep; the other two follow in increasing order. This
     * keeps the 2x2 system of the second operation well conditioned (its
     * determinant is ~ rotation angle times that component). */
    int perm[3];
    {
        int p = 0;
        for (int a = 1; a < 3; ++a)
            if (fabs(B[a]) > fabs(B[p])) p = a;
        int b, c;
        others(p, &b, &c);
        perm[0] = p; perm[1] = b; perm[2] = c;
    }
    /* M = P R P^T in the permuted frame, with its diagonal deviations Dd */
    double M[3][3], Dd[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j)
            M[i][j] = D[perm[i]][perm[j]] + (i == j ? 1.0 : 0.0);
        Dd[i] = D[perm[i]][perm[i]];
    }

    /* Reduce M to the identity by five row operations E1..E5 on rows 0, 1, 2,
     * 1, 0; then M = E1^-1 E2^-1 E3^-1 E4^-1 E5^-1 and the sweeps applied to
     * f are E5^-1 first, E1^-1 last. Each E = I + e_r c^T has inverse
     * I - e_r c^T, i.e. the sweep moves v_r by -c.v. */
    double ops[5][3]; /* per operation: coefficients on the three rows */
    int rows[5] = {0, 1, 2, 1, 0};
    /* E1 (row 0): make M00 = 1 with the least-norm combination of rows 1, 2 */
    {
        double den = M[1][0] * M[1][0] + M[2][0] * M[2][0];
        double a = 0.0, b = 0.0;
        if (den > 0.0) {
            a = -Dd[0] * M[1][0] / den;
            b = -Dd[0] * M[2][0] / den;
        }
        row_op(M, 0, 1, a, 2, b);
        Dd[0] = 0.0;
        M[0][0] = 1.0;
        ops[0][0] = 0.0; ops[0][1] = a; ops[0][2] = b;
    }
    /* E2 (row 1): make M10 = 0 and M11 = 1 with rows 0, 2 */
    {
        double det = M[2][1] - M[2][0] * M[0][1];
        double rhs0 = -M[1][0], rhs1 = -Dd[1];
        double c, d;
        if (det != 0.0) {
            /* c*M00 + d*M20 = rhs0 (M00 = 1); c*M01 + d*M21 = rhs1 */
            d = (rhs1 - M[0][1] * rhs0) / det;
            c = rhs0 - d * M[2][0];
        } else { /* R = I: the system is consistent with d = 0 */
            d = 0.0;
            c = rhs0;
        }
        row_op(M, 1, 0, c, 2, d);
        M[1][0] = 0.0;
        M[1][1] = 1.0;
        Dd[1] = 0.0;
        ops[1][0] = c; ops[1][1] = 0.0; ops[1][2] = d;
    }
    /* E3 (row 2): make M20 = M21 = 0 with rows 0, 1 */
    {
        double e = -M[2][0];
        double gq = -M[2][1] - e * M[0][1];
        row_op(M, 2, 0, e, 1, gq);
        ops[2][0] = e; ops[2][1] = gq; ops[2][2] = 0.0;
    }
    /* E4 (row 1): clear M12 with row 2 */
    {
        double c = -M[1][2];
        row_op(M, 1, 2, c, 0, 0.0);
        ops[3][0] = 0.0; ops[3][1] = 0.0; ops[3][2] = c;
    }
    /* E5 (row 0): clear M01, M02 with rows 1, 2 */
    {
        double a = -M[0][1], b = -M[0][2];
        row_op(M, 0, 1, a, 2, b);
        ops[4][0] = 0.0; ops[4][1] = a; ops[4][2] = b;
    }
    /* Sweep k (k = 0..4) is E_{5-k}^{-1}: row rows[4-k], coefficients -ops */
    double L[5][3][3]; /* linear part of each sweep, permuted frame */
    for (int k = 0; k < 5; ++k) {
        int op = 4 - k, r = rows[op];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) L[k][a][b] = (a == b) ? 1.0 : 0.0;
        for (int b = 0; b < 3; ++b)
            if (b != r) L[k][r][b] = -ops[op][b];
    }
    /* Constants: the translation goes into sweeps 2 (row 2), 3 (row 1) and 4
     * (row 0): b' = L4 L3 c2 e_2 + L4 c3 e_1 + c4 e_0 in the permuted frame. */
    double bp[3] = {bvec[perm[0]], bvec[perm[1]], bvec[perm[2]]};
    double K[3], Lv[3];
    {
        double tmp[3];
        for (int a = 0; a < 3; ++a) tmp[a] = L[3][a][2];
        for (int a = 0; a < 3; ++a) K[a] = L[4][a][0] * tmp[0] + L[4][a][1] * tmp[1] + L[4][a][2] * tmp[2];
        for (int a = 0; a < 3; ++a) Lv[a] = L[4][a][1];
    }
    double c2 = bp[2] / K[2];
    double c3 = (bp[1] - c2 * K[1]) / Lv[1];
    double c4 = bp[0] - c2 * K[0] - c3 * Lv[0];
    double consts[5] = {0.0, 0.0, c2, c3, c4};
    for (int k = 0; k < 5; ++k) {
        int r = rows[4 - k];
        int ax = perm[r], b, c;
        others(ax, &b, &c);
        /* permuted index of physical axes b and c */
        int pb = -1, pc = -1;
        for (int i = 0; i < 3; ++i) {
            if (perm[i] == b) pb = i;
            if (perm[i] == c) pc = i;
        }
        out[k * 4 + 0] = ax;
        out[k * 4 + 1] = L[k][r][pb];
        out[k * 4 + 2] = L[k][r][pc];
        out[k * 4 + 3] = consts[k];
    }
    return 0;
}

/* One zero-flux PFC sweep along velocity axis `axis` of one block, with
 * displacement coefb*v_b + coefc*v_c + cst (b < c the other two axes). */
static int sweep_block(double* blk, const or_species* sp, int axis,
                       double coefb, double coefc, double cst) {
    int nv0 = sp->nv[0], nv1 = sp->nv[1], nv2 = sp->nv[2];
    int n = sp->nv[axis];
    int b, c;
    others(axis, &b, &c);
    int nb = sp->nv[b], nc = sp->nv[c];
    long stride[3] = {1, nv0, (long)nv0 * nv1};
    (void)nv2;
    /* largest displacement over the block decides the ghost width */
    double amax = 0.0;
    for (int ib = 0; ib < nb; ++ib)
        for (int ic = 0; ic < nc; ++ic) {
            double d = fabs(coefb * vcentre(sp, b, ib) + coefc * vcentre(sp, c, ic) + cst) / sp->dv[axis];
            if (d > amax) amax = d;
        }
    int ng = (int)floor(amax) + 3;
    double* ext = (double*)calloc((size_t)(n + 2 * ng), sizeof(double));
    double* res = (double*)malloc(sizeof(double) * (size_t)n);
    for (int ib = 0; ib < nb; ++ib)
        for (int ic = 0; ic < nc; ++ic) {
            double disp = coefb * vcentre(sp, b, ib) + coefc * vcentre(sp, c, ic) + cst;
            double cc = disp / sp->dv[axis];
            long base = ib * stride[b] + ic * stride[c];
            for (int k = 0; k < n + 2 * ng; ++k) ext[k] = 0.0; /* zero ghosts */
            for (int k = 0; k < n; ++k) ext[ng + k] = blk[base + k * stride[axis]];
            if (or_pfc_line(ext, n, ng, cc, 1, res) != 0) {
                free(ext); free(res);
                return -2;
            }
            for (int k = 0; k < n; ++k) blk[base + k * stride[axis]] = res[k];
        }
    free(ext); free(res);
    return 0;
}

int or_advect_velocity(double* f, const or_grid* g, const or_species* sp,
                       const double* EB, double dt, int nshear) {
    long ncell = (long)g->nx * g->ny;
    long V = vblock(g, sp);
    double qm = sp->q / sp->m;
    if (g->nvdim == 1) {
        int n = sp->nv[0];
        int ng = 0;
        for (long cidx = 0; cidx < ncell; ++cidx) {
            int s = (int)floor(fabs(qm * EB[cidx * 6 + 0] * dt / sp->dv[0])) + 3;
            if (s > ng) ng = s;
        }
        double* ext = (double*)calloc((size_t)(n + 2 * ng), sizeof(double));
        double* res = (double*)malloc(sizeof(double) * (size_t)n);
        for (long cidx = 0; cidx < ncell; ++cidx) {
            double c = qm * EB[cidx * 6 + 0] * dt / sp->dv[0];
            for (int k = 0; k < n + 2 * ng; ++k) ext[k] = 0.0;
            for (int k = 0; k < n; ++k) ext[ng + k] = f[cidx * V + k];
            or_pfc_line(ext, n, ng, c, 1, res);
            for (int k = 0; k < n; ++k) f[cidx * V + k] = res[k];
        }
        free(ext); free(res);
        return 0;
    }
    for (long cidx = 0; cidx < ncell; ++cidx) {
        double sh[5 * 4];
        int rc = or_velocity_shears(qm, EB + cidx * 6, EB + cidx * 6 + 3, dt, nshear, sh);
        if (rc != 0) return rc;
        for (int k = 0; k < nshear; ++k) {
            rc = sweep_block(f + cidx * V, sp, (int)sh[k * 4 + 0], sh[k * 4 + 1],
                             sh[k * 4 + 2], sh[k * 4 + 3]);
            if (rc != 0) return rc;
        }
    }
    return 0;
}
