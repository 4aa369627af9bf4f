/*
 * Oracle: ten-moment Maxwellian, its discrete fit, and the exchange step of
 * moment fitting (test infrastructure only; see oracle.h).
 *
 * Paper Sec. 2.2 and Algorithm 1 ("Moment Fitting"): compute the ten-moment
 * Maxwellian f_M,V from the moments of f and f_M,F from the fluid moments
 * rescaled by n_V/n_F, exchange f <- f - f_M,V + f_M,F, then limit f by
 * clipping negative values and rescaling to the density before the exchange.
 *
 * The paper writes f_M with the continuous formula. The fit used here makes
 * the MIDPOINT moments of degree <= 2 of the sampled Maxwellian equal the
 * targets, so that the exchange changes the discrete moments of f by exactly
 * (fluid - Vlasov). It is solved by Newton's method on the natural
 * (exponential-family) parameters eta of
 *     M(v) = exp(eta . phi(w)),  w_a = (v_a - u0_a) / sigma_a,
 *     phi = (1, w_a, w_a w_b (a <= b)),
 * where u0 and sigma_a^2 = Theta0_aa come from the targets. The moment
 * equations D(eta) = T are the gradient of the convex function
 * L(eta) = sum_c M(v_c) dv^3 - eta . T, whose Hessian is the Gram matrix
 * J = sum_c M phi phi^T dv^3; steps are damped by backtracking on L.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define TWO_PI 6.283185307179586476925286766559

/* Cholesky of a d x d SPD matrix (row-major); returns 0 if PD. */
static int cholesky(const double* A, int d, double* L) {
    for (int i = 0; i < d * d; ++i) L[i] = 0.0;
    for (int i = 0; i < d; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = A[i * d + j];
            for (int k = 0; k < j; ++k) s -= L[i * d + k] * L[j * d + k];
            if (i == j) {
                if (!(s > 0.0)) return -1;
                L[i * d + i] = sqrt(s);
            } else {
                L[i * d + j] = s / L[j * d + j];
            }
        }
    return 0;
}

/* Inverse of an SPD d x d matrix via Gauss-Jordan (d <= 3). */
static int invert(const double* A, int d, double* Ainv) {
    double M[3][6];
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < 2 * d; ++j)
            M[i][j] = j < d ? A[i * d + j] : (j - d == i ? 1.0 : 0.0);
    for (int p = 0; p < d; ++p) {
        int piv = p;
        for (int r = p + 1; r < d; ++r)
            if (fabs(M[r][p]) > fabs(M[piv][p])) piv = r;
        if (M[piv][p] == 0.0) return -1;
        if (piv != p)
            for (int j = 0; j < 2 * d; ++j) { double t = M[p][j]; M[p][j] = M[piv][j]; M[piv][j] = t; }
        double inv = 1.0 / M[p][p];
        for (int j = 0; j < 2 * d; ++j) M[p][j] *= inv;
        for (int r = 0; r < d; ++r)
            if (r != p) {
                double fct = M[r][p];
                for (int j = 0; j < 2 * d; ++j) M[r][j] -= fct * M[p][j];
            }
    }
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) Ainv[i * d + j] = M[i][j + d];
    return 0;
}

static double det3(const double* A, int d) {
    if (d == 1) return A[0];
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}

/* Solve the n x n system A x = b by Gaussian elimination with partial
 * pivoting (A, b overwritten). Returns 0 on success. */
static int solve(double* A, double* b, int n, double* x) {
    for (int p = 0; p < n; ++p) {
        int piv = p;
        for (int r = p + 1; r < n; ++r)
            if (fabs(A[r * n + p]) > fabs(A[piv * n + p])) piv = r;
        if (!(fabs(A[piv * n + p]) > 0.0)) return -1;
        if (piv != p) {
            for (int j = 0; j < n; ++j) { double t = A[p * n + j]; A[p * n + j] = A[piv * n + j]; A[piv * n + j] = t; }
            double t = b[p]; b[p] = b[piv]; b[piv] = t;
        }
        for (int r = p + 1; r < n; ++r) {
            double fct = A[r * n + p] / A[p * n + p];
            for (int j = p; j < n; ++j) A[r * n + j] -= fct * A[p * n + j];
            b[r] -= fct * b[p];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int j = r + 1; j < n; ++j) s -= A[r * n + j] * x[j];
        x[r] = s / A[r * n + r];
    }
    return 0;
}

/* phi(w) for d = 1 (1, w, ww) or d = 3 (1, w_a, w_a w_b with a <= b in the
 * order xx, xy, xz, yy, yz, zz). Returns the number of functions. */
static int phi_eval(const double* w, int d, double* phi) {
    if (d == 1) {
        phi[0] = 1.0; phi[1] = w[0]; phi[2] = w[0] * w[0];
        return 3;
    }
    phi[0] = 1.0;
    phi[1] = w[0]; phi[2] = w[1]; phi[3] = w[2];
    phi[4] = w[0] * w[0]; phi[5] = w[0] * w[1]; phi[6] = w[0] * w[2];
    phi[7] = w[1] * w[1]; phi[8] = w[1] * w[2]; phi[9] = w[2] * w[2];
    return 10;
}

/* Symmetric d x d matrix from the 6 (or 1) packed second-order entries. */
static void unpack_sym(const double* p, int d, double* S) {
    if (d == 1) { S[0] = p[0]; return; }
    S[0] = p[0]; S[1] = p[1]; S[2] = p[2];
    S[3] = p[1]; S[4] = p[3]; S[5] = p[4];
    S[6] = p[2]; S[7] = p[4]; S[8] = p[5];
}

typedef struct {
    const or_species* sp;
    int d;
    double u0[3], sig[3];
    long npts;
    double vol; /* dv^d */
} fit_ctx;

static void grid_w(const fit_ctx* fc, long idx, double* w) {
    const or_species* sp = fc->sp;
    if (fc->d == 1) {
        double v = sp->vmin[0] + (idx + 0.5) * sp->dv[0];
        w[0] = (v - fc->u0[0]) / fc->sig[0];
        return;
    }
    long i = idx % sp->nv[0];
    long j = (idx / sp->nv[0]) % sp->nv[1];
    long k = idx / ((long)sp->nv[0] * sp->nv[1]);
    long ijk[3] = {i, j, k};
    for (int a = 0; a < 3; ++a) {
        double v = sp->vmin[a] + (ijk[a] + 0.5) * sp->dv[a];
        w[a] = (v - fc->u0[a]) / fc->sig[a];
    }
}

/* Discrete moments D (nphi) and, if J != NULL, the Gram matrix. */
static void discrete_moments(const fit_ctx* fc, const double* eta, int nphi,
                             double* D, double* J) {
    for (int a = 0; a < nphi; ++a) D[a] = 0.0;
    if (J) for (int a = 0; a < nphi * nphi; ++a) J[a] = 0.0;
    for (long c = 0; c < fc->npts; ++c) {
        double w[3], phi[10];
        grid_w(fc, c, w);
        phi_eval(w, fc->d, phi);
        double q = 0.0;
        for (int a = 0; a < nphi; ++a) q += eta[a] * phi[a];
        double M = exp(q) * fc->vol;
        for (int a = 0; a < nphi; ++a) D[a] += M * phi[a];
        if (J)
            for (int a = 0; a < nphi; ++a)
                for (int b = 0; b < nphi; ++b) J[a * nphi + b] += M * phi[a] * phi[b];
    }
}

int or_maxent_fit(const double* target, const or_species* sp, int nvdim,
                  double tol, int max_iter, double* theta, int* iters,
                  int* status) {
    int d = nvdim;
    int nphi = d == 1 ? 3 : 10;
    int ntheta = nphi;
    for (int a = 0; a < ntheta; ++a) theta[a] = 0.0;
    *iters = 0;
    double n = target[0];
    if (!(n > 0.0) || !isfinite(n)) { *status = 2; return 0; }

    /* targets -> u0, Theta0 (temperature over mass, Theta = k_B T / m) */
    fit_ctx fc;
    fc.sp = sp; fc.d = d;
    fc.npts = d == 1 ? sp->nv[0] : (long)sp->nv[0] * sp->nv[1] * sp->nv[2];
    fc.vol = d == 1 ? sp->dv[0] : sp->dv[0] * sp->dv[1] * sp->dv[2];
    double Th0[9], E2[9];
    for (int a = 0; a < d; ++a) fc.u0[a] = target[1 + a] / n;
    unpack_sym(target + 1 + d, d, E2);
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) Th0[a * d + b] = E2[a * d + b] / n - fc.u0[a] * fc.u0[b];
    double Lc[9];
    if (cholesky(Th0, d, Lc) != 0) { *status = 2; return 0; }
    for (int a = 0; a < d; ++a) fc.sig[a] = sqrt(Th0[a * d + a]);

    /* continuous Maxwellian of the targets: the fallback and the start */
    double cont[10];
    cont[0] = n;
    for (int a = 0; a < d; ++a) cont[1 + a] = fc.u0[a];
    if (d == 1) cont[2] = Th0[0];
    else {
        cont[4] = Th0[0]; cont[5] = Th0[1]; cont[6] = Th0[2];
        cont[7] = Th0[4]; cont[8] = Th0[5]; cont[9] = Th0[8];
    }

    /* targets in phi-space: (n, 0, n * correlation) */
    double T[10], Corr[9], P[9];
    T[0] = n;
    for (int a = 0; a < d; ++a) T[1 + a] = 0.0;
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) Corr[a * d + b] = Th0[a * d + b] / (fc.sig[a] * fc.sig[b]);
    if (d == 1) T[2] = n;
    else {
        T[4] = n * Corr[0]; T[5] = n * Corr[1]; T[6] = n * Corr[2];
        T[7] = n * Corr[4]; T[8] = n * Corr[5]; T[9] = n * Corr[8];
    }
    if (invert(Corr, d, P) != 0) { *status = 2; return 0; }

    /* eta of the continuous Maxwellian */
    double eta[10];
    eta[0] = log(n) - 0.5 * d * log(TWO_PI) - 0.5 * log(det3(Th0, d));
    for (int a = 0; a < d; ++a) eta[1 + a] = 0.0;
    if (d == 1) eta[2] = -0.5 * P[0];
    else {
        eta[4] = -0.5 * P[0]; eta[5] = -P[1]; eta[6] = -P[2];
        eta[7] = -0.5 * P[4]; eta[8] = -P[5]; eta[9] = -0.5 * P[8];
    }

    int converged = 0, it = 0;
    double D[10], J[100], G[10], delta[10], rhs[10];
    for (it = 0; it <= max_iter; ++it) {
        discrete_moments(&fc, eta, nphi, D, J);
        double gmax = 0.0;
        for (int a = 0; a < nphi; ++a) {
            G[a] = D[a] - T[a];
            if (fabs(G[a]) > gmax || !isfinite(G[a])) gmax = isfinite(G[a]) ? fabs(G[a]) : INFINITY;
        }
        if (gmax <= tol * n) { converged = 1; break; }
        if (!isfinite(gmax) || it == max_iter) break;
        for (int a = 0; a < nphi; ++a) rhs[a] = -G[a];
        if (solve(J, rhs, nphi, delta) != 0) break;
        /* damped step: backtracking on L(eta) = D_0(eta) - eta.T unless the
         * residual is already small (then the full Newton step is taken) */
        double lam = 1.0;
        if (gmax > 1e-6 * n) {
            double L0 = D[0], gd = 0.0;
            for (int a = 0; a < nphi; ++a) { L0 -= eta[a] * T[a]; gd += G[a] * delta[a]; }
            for (int k = 0; k < 40; ++k) {
                double et[10], Dt[10];
                for (int a = 0; a < nphi; ++a) et[a] = eta[a] + lam * delta[a];
                discrete_moments(&fc, et, nphi, Dt, NULL);
                double L1 = Dt[0];
                for (int a = 0; a < nphi; ++a) L1 -= et[a] * T[a];
                if (isfinite(L1) && L1 <= L0 + 1e-4 * lam * gd) break;
                lam *= 0.5;
            }
        }
        for (int a = 0; a < nphi; ++a) eta[a] += lam * delta[a];
    }
    *iters = it;

    if (converged) {
        /* eta -> theta: Theta_w = (-2 mu)^-1, u_w = Theta_w lambda */
        double mu[9], negmu2[9], Thw[9], Lw[9];
        double lamv[3];
        for (int a = 0; a < d; ++a) lamv[a] = eta[1 + a];
        if (d == 1) mu[0] = eta[2];
        else {
            mu[0] = eta[4]; mu[1] = 0.5 * eta[5]; mu[2] = 0.5 * eta[6];
            mu[3] = mu[1]; mu[4] = eta[7]; mu[5] = 0.5 * eta[8];
            mu[6] = mu[2]; mu[7] = mu[5]; mu[8] = eta[9];
        }
        for (int a = 0; a < d * d; ++a) negmu2[a] = -2.0 * mu[a];
        if (cholesky(negmu2, d, Lw) == 0 && invert(negmu2, d, Thw) == 0) {
            double uw[3], quad = 0.0, detD = 1.0;
            for (int a = 0; a < d; ++a) {
                uw[a] = 0.0;
                for (int b = 0; b < d; ++b) uw[a] += Thw[a * d + b] * lamv[b];
            }
            for (int a = 0; a < d; ++a) quad += lamv[a] * uw[a];
            for (int a = 0; a < d; ++a) detD *= fc.sig[a];
            double nprime = exp(eta[0] + 0.5 * quad) * pow(TWO_PI, 0.5 * d) *
                            sqrt(det3(Thw, d)) * detD;
            theta[0] = nprime;
            for (int a = 0; a < d; ++a) theta[1 + a] = fc.u0[a] + fc.sig[a] * uw[a];
            if (d == 1) theta[2] = fc.sig[0] * fc.sig[0] * Thw[0];
            else {
                int pk = 4;
                for (int a = 0; a < 3; ++a)
                    for (int b = a; b < 3; ++b) theta[pk++] = fc.sig[a] * fc.sig[b] * Thw[a * 3 + b];
            }
            *status = 0;
            return 0;
        }
    }
    for (int a = 0; a < ntheta; ++a) theta[a] = cont[a];
    *status = 1;
    return 0;
}

void or_maxwellian_grid(const double* theta, const or_species* sp, int nvdim,
                        double* out) {
    int d = nvdim;
    long npts = d == 1 ? sp->nv[0] : (long)sp->nv[0] * sp->nv[1] * sp->nv[2];
    double n = theta[0], Th[9], Thi[9];
    if (!(n > 0.0)) {
        for (long c = 0; c < npts; ++c) out[c] = 0.0;
        return;
    }
    unpack_sym(theta + 1 + d, d, Th);
    invert(Th, d, Thi);
    double norm = n * pow(TWO_PI, -0.5 * d) / sqrt(det3(Th, d));
    for (long c = 0; c < npts; ++c) {
        double dvv[3];
        if (d == 1) {
            dvv[0] = sp->vmin[0] + (c + 0.5) * sp->dv[0] - theta[1];
        } else {
            long i = c % sp->nv[0];
            long j = (c / sp->nv[0]) % sp->nv[1];
            long k = c / ((long)sp->nv[0] * sp->nv[1]);
            long ijk[3] = {i, j, k};
            for (int a = 0; a < 3; ++a) dvv[a] = sp->vmin[a] + (ijk[a] + 0.5) * sp->dv[a] - theta[1 + a];
        }
        double q = 0.0;
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) q += dvv[a] * Thi[a * d + b] * dvv[b];
        out[c] = norm * exp(-0.5 * q);
    }
}

int or_moment_fit(double* f, const or_grid* g, const or_species* sp,
                  double* fluid, double tol, int max_iter, long* stats) {
    int d = g->nvdim;
    int ncomp = d == 1 ? 3 : 10;
    int nmom = d == 1 ? 4 : 20;
    long ncell = (long)g->nx * g->ny;
    long V = d == 1 ? sp->nv[0] : (long)sp->nv[0] * sp->nv[1] * sp->nv[2];
    double vol = d == 1 ? sp->dv[0] : sp->dv[0] * sp->dv[1] * sp->dv[2];
    double* mom = (double*)malloc(sizeof(double) * (size_t)(ncell * nmom));
    double* MV = (double*)malloc(sizeof(double) * (size_t)V);
    double* MF = (double*)malloc(sizeof(double) * (size_t)V);
    or_moments(f, g, sp, mom);
    for (long c = 0; c < ncell; ++c) {
        double tV[10], tF[10], thV[10], thF[10];
        for (int a = 0; a < ncomp; ++a) tV[a] = mom[c * nmom + a];
        double nV = tV[0], nF = fluid[c * ncomp + 0];
        double scale = nF > 0.0 ? nV / nF : 0.0;
        for (int a = 0; a < ncomp; ++a) tF[a] = fluid[c * ncomp + a] * scale;
        int itV, itF, stV, stF;
        or_maxent_fit(tV, sp, d, tol, max_iter, thV, &itV, &stV);
        or_maxent_fit(tF, sp, d, tol, max_iter, thF, &itF, &stF);
        stats[0] += itV + itF;
        stats[1] += (stV == 1) + (stF == 1);
        for (int a = 0; a < ncomp; ++a) fluid[c * ncomp + a] = tF[a];
        if (stV == 2 || stF == 2) continue;
        or_maxwellian_grid(thV, sp, d, MV);
        or_maxwellian_grid(thF, sp, d, MF);
        double* fc = f + c * V;
        int neg = 0;
        for (long k = 0; k < V; ++k) {
            fc[k] = fc[k] - MV[k] + MF[k];
            if (fc[k] < 0.0) neg = 1;
        }
        if (neg) {
            double sum = 0.0;
            for (long k = 0; k < V; ++k) {
                if (fc[k] < 0.0) fc[k] = 0.0;
                sum += fc[k];
            }
            sum *= vol;
            double r = sum > 0.0 ? nV / sum : 0.0;
            for (long k = 0; k < V; ++k) fc[k] *= r;
            stats[2] += 1;
        }
    }
    free(mom); free(MV); free(MF);
    return 0;
}
