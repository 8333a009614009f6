/*
 * lasto_oracle.c -- plain FP64 CPU oracle of the LASTO interstitial Poisson step.
 *
 * TEST INFRASTRUCTURE ONLY (see lasto_oracle.h): loaded by the tests, the smoke
 * check and the benchmark's CPU baseline, never by the CUDA library.
 *
 * Written from the paper's Sections 1-3: the pseudo-density swap inside the
 * spheres (Section 1, Section 3 with the constraints beside Eq. 3.2-3.3), the
 * finite-difference / multigrid solve between the spheres (Section 3), the
 * Dirichlet data on the box edge (Eq. 2.7 via the exterior multipole expansion)
 * and the surface projection V_LM(R_i) of Eq. 3.6.  The readings taken where the
 * paper is silent are stated at each routine.
 */
#include "lasto_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#else
static int omp_get_max_threads(void) { return 1; }
static int omp_get_thread_num(void) { return 0; }
#endif

static const double PI = 3.14159265358979323846;

#define IDX(i, j, k, nx, ny) (((size_t)(k) * (size_t)(ny) + (size_t)(j)) * (size_t)(nx) + (size_t)(i))

/* ------------------------------------------------------------------ harmonics */
/* Real spherical harmonics of Eq. 3.1, written as solid harmonics r^l y_lm.  The
 * paper names "real spherical harmonics" without a convention; the reading is the
 * orthonormal set without Condon-Shortley phase, m > 0 ~ cos(m phi), m < 0 ~
 * sin(|m| phi). */
void or_solid_harmonics(double x, double y, double z, double* S)
{
    const double x2 = x * x, y2 = y * y, z2 = z * z, r2 = x2 + y2 + z2;
    S[0] = 0.5 * sqrt(1.0 / PI);
    const double c1 = sqrt(3.0 / (4.0 * PI));
    S[1] = c1 * y;
    S[2] = c1 * z;
    S[3] = c1 * x;
    S[4] = 0.5 * sqrt(15.0 / PI) * x * y;
    S[5] = 0.5 * sqrt(15.0 / PI) * y * z;
    S[6] = 0.25 * sqrt(5.0 / PI) * (3.0 * z2 - r2);
    S[7] = 0.5 * sqrt(15.0 / PI) * x * z;
    S[8] = 0.25 * sqrt(15.0 / PI) * (x2 - y2);
    S[9] = 0.25 * sqrt(35.0 / (2.0 * PI)) * (3.0 * x2 - y2) * y;
    S[10] = 0.5 * sqrt(105.0 / PI) * x * y * z;
    S[11] = 0.25 * sqrt(21.0 / (2.0 * PI)) * y * (5.0 * z2 - r2);
    S[12] = 0.25 * sqrt(7.0 / PI) * z * (5.0 * z2 - 3.0 * r2);
    S[13] = 0.25 * sqrt(21.0 / (2.0 * PI)) * x * (5.0 * z2 - r2);
    S[14] = 0.25 * sqrt(105.0 / PI) * (x2 - y2) * z;
    S[15] = 0.25 * sqrt(35.0 / (2.0 * PI)) * (x2 - 3.0 * y2) * x;
    S[16] = 0.75 * sqrt(35.0 / PI) * x * y * (x2 - y2);
    S[17] = 0.75 * sqrt(35.0 / (2.0 * PI)) * (3.0 * x2 - y2) * y * z;
    S[18] = 0.75 * sqrt(5.0 / PI) * x * y * (7.0 * z2 - r2);
    S[19] = 0.75 * sqrt(5.0 / (2.0 * PI)) * y * z * (7.0 * z2 - 3.0 * r2);
    S[20] = (3.0 / 16.0) * sqrt(1.0 / PI) * (35.0 * z2 * z2 - 30.0 * z2 * r2 + 3.0 * r2 * r2);
    S[21] = 0.75 * sqrt(5.0 / (2.0 * PI)) * x * z * (7.0 * z2 - 3.0 * r2);
    S[22] = (3.0 / 8.0) * sqrt(5.0 / PI) * (x2 - y2) * (7.0 * z2 - r2);
    S[23] = 0.75 * sqrt(35.0 / (2.0 * PI)) * (x2 - 3.0 * y2) * x * z;
    S[24] = (3.0 / 16.0) * sqrt(35.0 / PI) * (x2 * (x2 - 3.0 * y2) - y2 * (3.0 * x2 - y2));
}

static int l_of(int lm) { return lm >= 16 ? 4 : lm >= 9 ? 3 : lm >= 4 ? 2 : lm >= 1 ? 1 : 0; }

/* ------------------------------------------------------------------ quadrature */
/* Gauss-Legendre nodes by Newton's method on P_n (three-term recurrence). */
int or_gauss_legendre(int n, double* t, double* w)
{
    if (n < 1) return OR_INVALID_ARG;
    for (int i = 0; i < n; i++) {
        double z = cos(PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = (n == 1) ? 1.0 : n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = (n == 1) ? 1.0 : n * (z * p1 - p0) / (z * z - 1.0);
        }
        t[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ mesh */
/* Section 3: "fine meshes near the atoms and coarse meshes at large distances".
 * Reading: a symmetric power-law grading per axis (formula in the header). */
int or_mesh_axis(int n, double c, double L, double h_min, double h_max, double p_max, double* x, double* info)
{
    if (n < 3 || (n - 1) % 2 != 0 || !(L > 0.0) || !(h_min > 0.0)) return OR_INVALID_ARG;
    const double m = 0.5 * (n - 1);
    double A = h_min * m, B = L - A, p = 1.0;
    if (B < -1e-12 * L) return OR_INVALID_ARG;      /* centre spacing too wide for the box */
    if (B <= 1e-12 * L) { A = L; B = 0.0; }         /* uniform */
    else {
        p = (h_max * m - A) / B;
        if (p > p_max) {
            p = p_max;
            B = (h_max * m - L) / (p_max - 1.0);
            A = L - B;
        }
        if (!(p >= 1.0) || !(A > 0.0)) return OR_INVALID_ARG;
    }
    for (int i = 0; i < n; i++) {
        double xi = (i - m) / m;
        double g = (B == 0.0) ? 0.0 : B * pow(fabs(xi), p);
        x[i] = c + A * xi + (xi < 0.0 ? -g : g);
    }
    x[0] = c - L;
    x[n - 1] = c + L;
    if (info) {
        int im = (int)m;
        info[0] = A; info[1] = B; info[2] = p;
        info[3] = x[im + 1] - x[im];
        info[4] = x[n - 1] - x[n - 2];
    }
    return OR_OK;
}

void or_dual_lengths(int n, const double* x, double* v)
{
    v[0] = 0.5 * (x[1] - x[0]);
    v[n - 1] = 0.5 * (x[n - 1] - x[n - 2]);
    for (int i = 1; i < n - 1; i++) v[i] = 0.5 * (x[i + 1] - x[i - 1]);
}

/* ------------------------------------------------------------------ density model */
/* Normalised Slater exponential zeta^3/(8 pi) e^{-zeta r}: integrates to one electron. */
static double slater(double zeta, double r) { return zeta * zeta * zeta / (8.0 * PI) * exp(-zeta * r); }

/* n_e(x) = sum_j [ sum_k w_jk slater(zeta_jk, r_j) + rho_ns,j(x) ].
 * Reading of the nonspherical part (the paper's densities are not available):
 * rho_ns,j = slater(zeta_j1, r) (1 - r^2/R^2)^2 sum_{l=1..4,m} c_lm (r/R)^l y_lm, zero
 * for r >= R_j: smooth, confined to its own sphere, no monopole. */
double or_density(int na, const double* pos, const double* R, const double* w, const double* zeta,
                  const double* clm, double x, double y, double z)
{
    double s = 0.0;
    for (int j = 0; j < na; j++) {
        const double dx = x - pos[3 * j], dy = y - pos[3 * j + 1], dz = z - pos[3 * j + 2];
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        for (int k = 0; k < 3; k++) s += w[3 * j + k] * slater(zeta[3 * j + k], r);
        const double Rj = R[j];
        if (r < Rj) {
            const double t = 1.0 - r * r / (Rj * Rj);
            const double f = slater(zeta[3 * j], r) * t * t;
            double S[25];
            or_solid_harmonics(dx, dy, dz, S);
            double ang = 0.0;
            for (int lm = 1; lm < 25; lm++) ang += clm[24 * j + lm - 1] * S[lm] / pow(Rj, l_of(lm));
            s += f * ang;
        }
    }
    return s;
}

void or_density_grid(int na, const double* pos, const double* R, const double* w, const double* zeta,
                     const double* clm, int nx, int ny, int nz, const double* x, const double* y,
                     const double* z, double* out)
{
#pragma omp parallel for schedule(dynamic)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++)
                out[IDX(i, j, k, nx, ny)] = or_density(na, pos, R, w, zeta, clm, x[i], y[j], z[k]);
}

/* Spherical average of e^{-zeta |x - D|} over the sphere |x| = r, for a centre at
 * distance D > r:  (1/2rD) int_{|r-D|}^{r+D} e^{-zeta s} s ds, written out. */
static double sph_avg(double zeta, double r, double D)
{
    if (r < 1e-4) {  /* mean-value expansion: f(0) + r^2/6 Lap f(0) */
        return exp(-zeta * D) * (1.0 + r * r / 6.0 * (zeta * zeta - 2.0 * zeta / D));
    }
    const double a = fabs(r - D), b = r + D;
    return ((1.0 + zeta * a) * exp(-zeta * a) - (1.0 + zeta * b) * exp(-zeta * b)) / (2.0 * r * D * zeta * zeta);
}

static double sph_avg_dr(double zeta, double r, double D)
{
    if (r < 1e-4) return exp(-zeta * D) * r / 3.0 * (zeta * zeta - 2.0 * zeta / D);
    const double a = fabs(r - D), b = r + D;
    const double F = ((1.0 + zeta * a) * exp(-zeta * a) - (1.0 + zeta * b) * exp(-zeta * b)) / (2.0 * D * zeta * zeta);
    const double dF = (-(r - D) * exp(-zeta * a) + b * exp(-zeta * b)) / (2.0 * D);
    return dF / r - F / (r * r);
}

/* rho0_i(r): the monopole of n_e about atom i.  Own Slater terms are spherical;
 * neighbours' Slater terms enter through their spherical averages; the l >= 1
 * parts have no monopole and the neighbours' nonspherical parts vanish inside
 * sphere i (spheres do not overlap). */
void or_monopole(int na, const double* pos, const double* w, const double* zeta, int i, double r,
                 double* rho0, double* drho0)
{
    double s = 0.0, ds = 0.0;
    for (int k = 0; k < 3; k++) {
        const double g = w[3 * i + k] * slater(zeta[3 * i + k], r);
        s += g;
        ds += -zeta[3 * i + k] * g;
    }
    for (int j = 0; j < na; j++) {
        if (j == i) continue;
        const double dx = pos[3 * j] - pos[3 * i], dy = pos[3 * j + 1] - pos[3 * i + 1], dz = pos[3 * j + 2] - pos[3 * i + 2];
        const double D = sqrt(dx * dx + dy * dy + dz * dz);
        for (int k = 0; k < 3; k++) {
            const double zt = zeta[3 * j + k];
            const double c = w[3 * j + k] * zt * zt * zt / (8.0 * PI);
            s += c * sph_avg(zt, r, D);
            ds += c * sph_avg_dr(zt, r, D);
        }
    }
    *rho0 = s;
    *drho0 = ds;
}

/* Solve a 3x3 system by Gaussian elimination with partial pivoting. */
static int solve3(double M[3][3], double rhs[3], double out[3])
{
    int p[3] = {0, 1, 2};
    for (int c = 0; c < 3; c++) {
        int best = c;
        for (int r = c + 1; r < 3; r++)
            if (fabs(M[p[r]][c]) > fabs(M[p[best]][c])) best = r;
        int t = p[c]; p[c] = p[best]; p[best] = t;
        if (M[p[c]][c] == 0.0) return OR_INVALID_ARG;
        for (int r = c + 1; r < 3; r++) {
            double f = M[p[r]][c] / M[p[c]][c];
            for (int cc = c; cc < 3; cc++) M[p[r]][cc] -= f * M[p[c]][cc];
            rhs[p[r]] -= f * rhs[p[c]];
        }
    }
    for (int c = 2; c >= 0; c--) {
        double s = rhs[p[c]];
        for (int cc = c + 1; cc < 3; cc++) s -= M[p[c]][cc] * out[cc];
        out[c] = s / M[p[c]][c];
    }
    return OR_OK;
}

/* Section 3, constraints beside Eq. 3.2-3.3: the pseudo-density carries the same
 * charge q as rho - Z delta inside the sphere, and meets rho in value and slope at
 * R.  Reading of the garbled charge condition: 4 pi int_0^R rho_tilde r^2 dr =
 * 4 pi int_0^R rho0 r^2 dr - Z.  Reading of the shape (the paper gives only the
 * three constraints): the even quartic a + b r^2 + c r^4.  The charge integral
 * uses 64-point Gauss-Legendre on [0, R]. */
void or_sphere_params(int na, const double* pos, const double* Z, const double* R, const double* w,
                      const double* zeta, double* q, double* rhoR, double* drhoR, double* coef)
{
    double t[64], wt[64];
    or_gauss_legendre(64, t, wt);
    for (int i = 0; i < na; i++) {
        const double Ri = R[i];
        double acc = 0.0;
        for (int g = 0; g < 64; g++) {
            const double r = 0.5 * Ri * (t[g] + 1.0);
            double rho, drho;
            or_monopole(na, pos, w, zeta, i, r, &rho, &drho);
            acc += 0.5 * Ri * wt[g] * rho * r * r;
        }
        q[i] = 4.0 * PI * acc - Z[i];
        or_monopole(na, pos, w, zeta, i, Ri, &rhoR[i], &drhoR[i]);
        double M[3][3] = {{4.0 * PI * pow(Ri, 3) / 3.0, 4.0 * PI * pow(Ri, 5) / 5.0, 4.0 * PI * pow(Ri, 7) / 7.0},
                          {1.0, Ri * Ri, pow(Ri, 4)},
                          {0.0, 2.0 * Ri, 4.0 * pow(Ri, 3)}};
        double rhs[3] = {q[i], rhoR[i], drhoR[i]};
        solve3(M, rhs, &coef[3 * i]);
    }
}

/* ------------------------------------------------------------------ deposit */
int or_deposit(int na, const double* pos, const double* Z, const double* R, const double* w,
               const double* zeta, const double* clm, int nx, int ny, int nz, const double* x,
               const double* y, const double* z, double* b, int* owner)
{
    double* q = malloc(sizeof(double) * na);
    double* rhoR = malloc(sizeof(double) * na);
    double* drhoR = malloc(sizeof(double) * na);
    double* coef = malloc(sizeof(double) * 3 * na);
    or_sphere_params(na, pos, Z, R, w, zeta, q, rhoR, drhoR, coef);
#pragma omp parallel for schedule(dynamic)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                int own = -1;
                double r = 0.0;
                for (int a = 0; a < na; a++) {
                    const double dx = x[i] - pos[3 * a], dy = y[j] - pos[3 * a + 1], dz = z[k] - pos[3 * a + 2];
                    const double ra = sqrt(dx * dx + dy * dy + dz * dz);
                    if (ra < R[a]) { own = a; r = ra; break; }
                }
                double val = or_density(na, pos, R, w, zeta, clm, x[i], y[j], z[k]);
                if (own >= 0) {
                    double rho0, drho0;
                    or_monopole(na, pos, w, zeta, own, r, &rho0, &drho0);
                    const double* c = &coef[3 * own];
                    val = val - rho0 + (c[0] + c[1] * r * r + c[2] * r * r * r * r);
                }
                b[IDX(i, j, k, nx, ny)] = 4.0 * PI * val;
                if (owner) owner[IDX(i, j, k, nx, ny)] = own;
            }
    free(q); free(rhoR); free(drhoR); free(coef);
    return OR_OK;
}

/* ------------------------------------------------------------------ boundary data */
void or_multipoles(int nx, int ny, int nz, const double* x, const double* y, const double* z,
                   const double* b, double cx, double cy, double cz, double* Q)
{
    double* vx = malloc(sizeof(double) * nx);
    double* vy = malloc(sizeof(double) * ny);
    double* vz = malloc(sizeof(double) * nz);
    or_dual_lengths(nx, x, vx);
    or_dual_lengths(ny, y, vy);
    or_dual_lengths(nz, z, vz);
    double* part = calloc((size_t)nz * 25, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++) {
        double S[25];
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                const double rho = b[IDX(i, j, k, nx, ny)] / (4.0 * PI);
                const double vol = vx[i] * vy[j] * vz[k];
                or_solid_harmonics(x[i] - cx, y[j] - cy, z[k] - cz, S);
                for (int lm = 0; lm < 25; lm++) part[25 * k + lm] += rho * vol * S[lm];
            }
    }
    for (int lm = 0; lm < 25; lm++) {
        double s = 0.0;
        for (int k = 0; k < nz; k++) s += part[25 * k + lm];
        Q[lm] = s;
    }
    free(part); free(vx); free(vy); free(vz);
}

static double multipole_potential(const double* Q, double dx, double dy, double dz)
{
    double S[25];
    or_solid_harmonics(dx, dy, dz, S);
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    double u = 0.0;
    for (int lm = 0; lm < 25; lm++) {
        const int l = l_of(lm);
        u -= 4.0 * PI / (2.0 * l + 1.0) * Q[lm] * S[lm] / pow(r, 2 * l + 1);
    }
    return u;
}

void or_boundary_fill(int nx, int ny, int nz, const double* x, const double* y, const double* z,
                      double cx, double cy, double cz, const double* Q, double* u)
{
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                if (i == 0 || j == 0 || k == 0 || i == nx - 1 || j == ny - 1 || k == nz - 1)
                    u[IDX(i, j, k, nx, ny)] = multipole_potential(Q, x[i] - cx, y[j] - cy, z[k] - cz);
            }
}

/* Exact superposition Dirichlet values (the alternative to Eq. 3.3's zero and to the
 * truncated multipole expansion): on each face node the continuum potential of the density
 * model, atom by atom, valid outside every sphere:
 *   Phi_j(r) = Z_j/r - sum_k w_k [1/r - e^{-zeta_k r}(1/r + zeta_k/2)]
 *              - sum_{l>=1,m} 4pi/(2l+1) c_lm M_l y_lm(r^) / r^(l+1),
 * the normalised-exponential potential of each Slater shell and the exterior multipoles of
 * the atom's nonspherical part, M_l = int_0^R zeta_1^3/(8pi) e^{-zeta_1 r}(1 - r^2/R^2)^2
 * (r/R)^l r^(l+2) dr (64-point Gauss-Legendre).  Writes only the six faces of u. */
void or_boundary_exact(int na, const double* pos, const double* Z, const double* R, const double* w,
                       const double* zeta, const double* clm, int nx, int ny, int nz, const double* x,
                       const double* y, const double* z, double* u)
{
    double* M = malloc(sizeof(double) * 5 * (na > 0 ? na : 1));
    double t[64], wt[64];
    or_gauss_legendre(64, t, wt);
    for (int j = 0; j < na; j++) {
        const double Rj = R[j], z1 = zeta[3 * j];
        for (int l = 0; l < 5; l++) {
            double s = 0.0;
            for (int q = 0; q < 64; q++) {
                const double r = 0.5 * Rj * (t[q] + 1.0), tt = 1.0 - r * r / (Rj * Rj);
                s += 0.5 * Rj * wt[q] * slater(z1, r) * tt * tt * pow(r / Rj, l) * pow(r, l + 2);
            }
            M[5 * j + l] = s;
        }
    }
#pragma omp parallel for schedule(dynamic)
    for (int k = 0; k < nz; k++)
        for (int jj = 0; jj < ny; jj++)
            for (int i = 0; i < nx; i++) {
                if (!(i == 0 || jj == 0 || k == 0 || i == nx - 1 || jj == ny - 1 || k == nz - 1)) continue;
                double v = 0.0;
                for (int j = 0; j < na; j++) {
                    const double dx = x[i] - pos[3 * j], dy = y[jj] - pos[3 * j + 1], dz = z[k] - pos[3 * j + 2];
                    const double r = sqrt(dx * dx + dy * dy + dz * dz);
                    v += Z[j] / r;
                    for (int q = 0; q < 3; q++) {
                        const double zq = zeta[3 * j + q];
                        v -= w[3 * j + q] * (1.0 / r - exp(-zq * r) * (1.0 / r + 0.5 * zq));
                    }
                    double S[25];
                    or_solid_harmonics(dx, dy, dz, S);
                    for (int lm = 1; lm < 25; lm++) {
                        const int l = l_of(lm);
                        v -= 4.0 * PI / (2 * l + 1) * clm[24 * j + lm - 1] * M[5 * j + l] * S[lm] / pow(r, 2 * l + 1);
                    }
                }
                u[IDX(i, jj, k, nx, ny)] = v;
            }
    free(M);
}

/* ------------------------------------------------------------------ operator */
/* One axis of the 7-point Laplacian on a nonuniform mesh:
 * 2/(h- + h+) [ (u+ - uP)/h+ - (uP - u-)/h- ]. */
static double axis_term(const double* c, int i, double um, double uP, double up)
{
    const double hm = c[i] - c[i - 1], hp = c[i + 1] - c[i];
    return (2.0 / (hm + hp)) * ((up - uP) / hp - (uP - um) / hm);
}

void or_apply_A(int nx, int ny, int nz, const double* x, const double* y, const double* z,
                const double* u, double* Au)
{
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                const size_t P = IDX(i, j, k, nx, ny);
                if (i == 0 || j == 0 || k == 0 || i == nx - 1 || j == ny - 1 || k == nz - 1) { Au[P] = 0.0; continue; }
                const double uP = u[P];
                Au[P] = axis_term(x, i, u[P - 1], uP, u[P + 1])
                      + axis_term(y, j, u[P - nx], uP, u[P + nx])
                      + axis_term(z, k, u[P - (size_t)nx * ny], uP, u[P + (size_t)nx * ny]);
            }
}

void or_residual(int nx, int ny, int nz, const double* x, const double* y, const double* z,
                 const double* u, const double* b, double* r)
{
    or_apply_A(nx, ny, nz, x, y, z, u, r);
#pragma omp parallel for schedule(static)
    for (int k = 1; k < nz - 1; k++)
        for (int j = 1; j < ny - 1; j++)
            for (int i = 1; i < nx - 1; i++) {
                const size_t P = IDX(i, j, k, nx, ny);
                r[P] = b[P] - r[P];
            }
}

double or_norm2_interior(int nx, int ny, int nz, const double* r)
{
    double* part = calloc(nz, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int k = 1; k < nz - 1; k++) {
        double s = 0.0;
        for (int j = 1; j < ny - 1; j++)
            for (int i = 1; i < nx - 1; i++) {
                const double v = r[IDX(i, j, k, nx, ny)];
                s += v * v;
            }
        part[k] = s;
    }
    double s = 0.0;
    for (int k = 0; k < nz; k++) s += part[k];
    free(part);
    return sqrt(s);
}

/* Gauss-Seidel on one colour: solve the node's own equation for uP with the
 * neighbours held.  Nodes of one colour only couple to the other colour. */
void or_rbgs_half(int nx, int ny, int nz, const double* x, const double* y, const double* z,
                  double* u, const double* b, int colour)
{
#pragma omp parallel for schedule(static)
    for (int k = 1; k < nz - 1; k++)
        for (int j = 1; j < ny - 1; j++)
            for (int i = 1; i < nx - 1; i++) {
                if (((i + j + k) & 1) != colour) continue;
                const size_t P = IDX(i, j, k, nx, ny);
                const size_t sy = nx, sz = (size_t)nx * ny;
                const double hxm = x[i] - x[i - 1], hxp = x[i + 1] - x[i];
                const double hym = y[j] - y[j - 1], hyp = y[j + 1] - y[j];
                const double hzm = z[k] - z[k - 1], hzp = z[k + 1] - z[k];
                const double ax = 2.0 / (hxm + hxp), ay = 2.0 / (hym + hyp), az = 2.0 / (hzm + hzp);
                const double off = ax * (u[P + 1] / hxp + u[P - 1] / hxm)
                                 + ay * (u[P + sy] / hyp + u[P - sy] / hym)
                                 + az * (u[P + sz] / hzp + u[P - sz] / hzm);
                const double diag = ax * (1.0 / hxp + 1.0 / hxm) + ay * (1.0 / hyp + 1.0 / hym) + az * (1.0 / hzp + 1.0 / hzm);
                u[P] = (off - b[P]) / diag;
            }
}

/* ------------------------------------------------------------------ transfers */
/* Weight of coarse node I in the linear interpolation at fine node f (physical
 * coordinates; coarse node I sits at fine node 2I). */
static double interp_w(const double* xf, int f, int I)
{
    if (f == 2 * I) return 1.0;
    if (f == 2 * I - 1) return (xf[f] - xf[2 * I - 2]) / (xf[2 * I] - xf[2 * I - 2]);
    if (f == 2 * I + 1) return (xf[2 * I + 2] - xf[f]) / (xf[2 * I + 2] - xf[2 * I]);
    return 0.0;
}

void or_restrict(int nx, int ny, int nz, const double* x, const double* y, const double* z,
                 const double* r, double* bc)
{
    const int cx = (nx + 1) / 2, cy = (ny + 1) / 2, cz = (nz + 1) / 2;
    double* vx = malloc(sizeof(double) * nx);
    double* vy = malloc(sizeof(double) * ny);
    double* vz = malloc(sizeof(double) * nz);
    or_dual_lengths(nx, x, vx);
    or_dual_lengths(ny, y, vy);
    or_dual_lengths(nz, z, vz);
    /* coarse dual lengths from the coarse coordinates (every other fine node) */
    double* Vx = malloc(sizeof(double) * cx);
    double* Vy = malloc(sizeof(double) * cy);
    double* Vz = malloc(sizeof(double) * cz);
    {
        double* t = malloc(sizeof(double) * (cx > cy ? (cx > cz ? cx : cz) : (cy > cz ? cy : cz)));
        for (int I = 0; I < cx; I++) t[I] = x[2 * I];
        or_dual_lengths(cx, t, Vx);
        for (int I = 0; I < cy; I++) t[I] = y[2 * I];
        or_dual_lengths(cy, t, Vy);
        for (int I = 0; I < cz; I++) t[I] = z[2 * I];
        or_dual_lengths(cz, t, Vz);
        free(t);
    }
    memset(bc, 0, sizeof(double) * (size_t)cx * cy * cz);
#pragma omp parallel for schedule(static)
    for (int K = 1; K < cz - 1; K++)
        for (int J = 1; J < cy - 1; J++)
            for (int I = 1; I < cx - 1; I++) {
                double acc = 0.0;
                for (int c = -1; c <= 1; c++)
                    for (int bb = -1; bb <= 1; bb++)
                        for (int a = -1; a <= 1; a++) {
                            const int fi = 2 * I + a, fj = 2 * J + bb, fk = 2 * K + c;
                            const double wgt = interp_w(x, fi, I) * vx[fi] * interp_w(y, fj, J) * vy[fj]
                                             * interp_w(z, fk, K) * vz[fk];
                            acc += wgt * r[IDX(fi, fj, fk, nx, ny)];
                        }
                bc[IDX(I, J, K, cx, cy)] = acc / (Vx[I] * Vy[J] * Vz[K]);
            }
    free(vx); free(vy); free(vz); free(Vx); free(Vy); free(Vz);
}

void or_prolong_add(int nx, int ny, int nz, const double* x, const double* y, const double* z,
                    const double* ec, double* u)
{
    const int cx = (nx + 1) / 2, cy = (ny + 1) / 2;
#pragma omp parallel for schedule(static)
    for (int k = 1; k < nz - 1; k++)
        for (int j = 1; j < ny - 1; j++)
            for (int i = 1; i < nx - 1; i++) {
                double e = 0.0;
                for (int K = k / 2; K <= (k + 1) / 2; K++)
                    for (int J = j / 2; J <= (j + 1) / 2; J++)
                        for (int I = i / 2; I <= (i + 1) / 2; I++)
                            e += interp_w(x, i, I) * interp_w(y, j, J) * interp_w(z, k, K) * ec[IDX(I, J, K, cx, cy)];
                u[IDX(i, j, k, nx, ny)] += e;
            }
}

/* ------------------------------------------------------------------ coarse solve */
/* Dense matrix of the interior operator (zero boundary values), LU with partial
 * pivoting, forward/back substitution. */
typedef struct {
    int n[3], m;
    double* LU;
    int* piv;
} coarse_lu;

static int coarse_factor(coarse_lu* c, int nx, int ny, int nz, const double* x, const double* y, const double* z)
{
    const int mx = nx - 2, my = ny - 2, mz = nz - 2, m = mx * my * mz;
    c->n[0] = nx; c->n[1] = ny; c->n[2] = nz; c->m = m;
    c->LU = calloc((size_t)m * m, sizeof(double));
    c->piv = malloc(sizeof(int) * m);
    double* A = c->LU;
    const double* cs[3] = {x, y, z};
    for (int k = 1; k <= mz; k++)
        for (int j = 1; j <= my; j++)
            for (int i = 1; i <= mx; i++) {
                const int row = ((k - 1) * my + (j - 1)) * mx + (i - 1);
                const int idx[3] = {i, j, k}, mm[3] = {mx, my, mz};
                const int stride[3] = {1, mx, mx * my};
                for (int ax = 0; ax < 3; ax++) {
                    const double* c_ = cs[ax];
                    const int p = idx[ax];
                    const double hm = c_[p] - c_[p - 1], hp = c_[p + 1] - c_[p];
                    const double s = 2.0 / (hm + hp);
                    A[(size_t)row * m + row] -= s * (1.0 / hm + 1.0 / hp);
                    if (p - 1 >= 1) A[(size_t)row * m + row - stride[ax]] += s / hm;
                    if (p + 1 <= mm[ax]) A[(size_t)row * m + row + stride[ax]] += s / hp;
                }
            }
    for (int col = 0; col < m; col++) {
        int best = col;
        for (int r = col + 1; r < m; r++)
            if (fabs(A[(size_t)r * m + col]) > fabs(A[(size_t)best * m + col])) best = r;
        c->piv[col] = best;
        if (best != col)
            for (int cc = 0; cc < m; cc++) {
                double t = A[(size_t)col * m + cc];
                A[(size_t)col * m + cc] = A[(size_t)best * m + cc];
                A[(size_t)best * m + cc] = t;
            }
        const double d = A[(size_t)col * m + col];
        if (d == 0.0) return OR_INVALID_ARG;
        for (int r = col + 1; r < m; r++) {
            const double f = A[(size_t)r * m + col] / d;
            A[(size_t)r * m + col] = f;
            if (f != 0.0)
                for (int cc = col + 1; cc < m; cc++) A[(size_t)r * m + cc] -= f * A[(size_t)col * m + cc];
        }
    }
    return OR_OK;
}

static void coarse_apply(const coarse_lu* c, const double* b, double* e)
{
    const int nx = c->n[0], ny = c->n[1], nz = c->n[2], mx = nx - 2, my = ny - 2, m = c->m;
    double* v = malloc(sizeof(double) * m);
    for (int k = 1; k < nz - 1; k++)
        for (int j = 1; j < ny - 1; j++)
            for (int i = 1; i < nx - 1; i++) v[((k - 1) * my + (j - 1)) * mx + (i - 1)] = b[IDX(i, j, k, nx, ny)];
    for (int col = 0; col < m; col++) {
        const int p = c->piv[col];
        if (p != col) { double t = v[col]; v[col] = v[p]; v[p] = t; }
    }
    for (int r = 0; r < m; r++) {
        double s = v[r];
        for (int cc = 0; cc < r; cc++) s -= c->LU[(size_t)r * m + cc] * v[cc];
        v[r] = s;
    }
    for (int r = m - 1; r >= 0; r--) {
        double s = v[r];
        for (int cc = r + 1; cc < m; cc++) s -= c->LU[(size_t)r * m + cc] * v[cc];
        v[r] = s / c->LU[(size_t)r * m + r];
    }
    memset(e, 0, sizeof(double) * (size_t)nx * ny * nz);
    for (int k = 1; k < nz - 1; k++)
        for (int j = 1; j < ny - 1; j++)
            for (int i = 1; i < nx - 1; i++) e[IDX(i, j, k, nx, ny)] = v[((k - 1) * my + (j - 1)) * mx + (i - 1)];
    free(v);
}

int or_coarse_solve(int nx, int ny, int nz, const double* x, const double* y, const double* z,
                    const double* b, double* e)
{
    coarse_lu c;
    int st = coarse_factor(&c, nx, ny, nz, x, y, z);
    if (st == OR_OK) coarse_apply(&c, b, e);
    free(c.LU); free(c.piv);
    return st;
}

/* ------------------------------------------------------------------ multigrid */
int or_num_levels(int nx, int ny, int nz)
{
    int L = 1;
    while ((nx > 9 || ny > 9 || nz > 9) && (nx - 1) % 2 == 0 && (ny - 1) % 2 == 0 && (nz - 1) % 2 == 0 &&
           nx >= 5 && ny >= 5 && nz >= 5) {
        nx = (nx + 1) / 2; ny = (ny + 1) / 2; nz = (nz + 1) / 2;
        L++;
    }
    if (nx > 9 || ny > 9 || nz > 9) return -1;
    return L;
}

typedef struct {
    int n[3];
    double* c[3];
    double *u, *b, *r;
} level;

typedef struct {
    int L, nu1, nu2;
    level lv[20];
    coarse_lu lu;
} mg_ctx;

static void mg_cycle(mg_ctx* g, int l, int fcycle)
{
    level* v = &g->lv[l];
    const int nx = v->n[0], ny = v->n[1], nz = v->n[2];
    if (l == g->L - 1) {
        /* exact solve as a correction: u += A^-1 (b - A u); keeps Dirichlet faces */
        const size_t N = (size_t)nx * ny * nz;
        double* e = malloc(sizeof(double) * N);
        or_residual(nx, ny, nz, v->c[0], v->c[1], v->c[2], v->u, v->b, v->r);
        coarse_apply(&g->lu, v->r, e);
        for (size_t p = 0; p < N; p++) v->u[p] += e[p];
        free(e);
        return;
    }
    for (int s = 0; s < g->nu1; s++) {
        or_rbgs_half(nx, ny, nz, v->c[0], v->c[1], v->c[2], v->u, v->b, 0);
        or_rbgs_half(nx, ny, nz, v->c[0], v->c[1], v->c[2], v->u, v->b, 1);
    }
    or_residual(nx, ny, nz, v->c[0], v->c[1], v->c[2], v->u, v->b, v->r);
    level* w = &g->lv[l + 1];
    or_restrict(nx, ny, nz, v->c[0], v->c[1], v->c[2], v->r, w->b);
    memset(w->u, 0, sizeof(double) * (size_t)w->n[0] * w->n[1] * w->n[2]);
    mg_cycle(g, l + 1, fcycle);
    if (fcycle) mg_cycle(g, l + 1, 0);
    or_prolong_add(nx, ny, nz, v->c[0], v->c[1], v->c[2], w->u, v->u);
    for (int s = 0; s < g->nu2; s++) {
        or_rbgs_half(nx, ny, nz, v->c[0], v->c[1], v->c[2], v->u, v->b, 0);
        or_rbgs_half(nx, ny, nz, v->c[0], v->c[1], v->c[2], v->u, v->b, 1);
    }
}

int or_mg_solve(int nx, int ny, int nz, const double* x, const double* y, const double* z,
                const double* b, double* u, int nu1, int nu2, int n_f, double tol, int max_cycles,
                double* hist, int* cycles_out)
{
    const int L = or_num_levels(nx, ny, nz);
    if (L < 1) return OR_INVALID_ARG;
    mg_ctx g;
    memset(&g, 0, sizeof g);
    g.L = L; g.nu1 = nu1; g.nu2 = nu2;
    const size_t N0 = (size_t)nx * ny * nz;
    for (int l = 0; l < L; l++) {
        level* v = &g.lv[l];
        if (l == 0) {
            v->n[0] = nx; v->n[1] = ny; v->n[2] = nz;
            v->c[0] = malloc(sizeof(double) * nx); memcpy(v->c[0], x, sizeof(double) * nx);
            v->c[1] = malloc(sizeof(double) * ny); memcpy(v->c[1], y, sizeof(double) * ny);
            v->c[2] = malloc(sizeof(double) * nz); memcpy(v->c[2], z, sizeof(double) * nz);
            v->u = u;
            v->b = (double*)b;
        } else {
            level* f = &g.lv[l - 1];
            for (int a = 0; a < 3; a++) {
                v->n[a] = (f->n[a] + 1) / 2;
                v->c[a] = malloc(sizeof(double) * v->n[a]);
                for (int I = 0; I < v->n[a]; I++) v->c[a][I] = f->c[a][2 * I];
            }
            const size_t N = (size_t)v->n[0] * v->n[1] * v->n[2];
            v->u = calloc(N, sizeof(double));
            v->b = calloc(N, sizeof(double));
        }
        v->r = calloc((size_t)v->n[0] * v->n[1] * v->n[2], sizeof(double));
    }
    level* cl = &g.lv[L - 1];
    int st = coarse_factor(&g.lu, cl->n[0], cl->n[1], cl->n[2], cl->c[0], cl->c[1], cl->c[2]);
    if (st != OR_OK) return st;

    /* ||b_eff||: residual of the boundary values with a zero interior (the boundary
     * contribution moved into b). */
    double* u0 = malloc(sizeof(double) * N0);
    memcpy(u0, u, sizeof(double) * N0);
    for (int k = 1; k < nz - 1; k++)
        for (int j = 1; j < ny - 1; j++)
            for (int i = 1; i < nx - 1; i++) u0[IDX(i, j, k, nx, ny)] = 0.0;
    level* f0 = &g.lv[0];
    or_residual(nx, ny, nz, x, y, z, u0, b, f0->r);
    const double bnorm = or_norm2_interior(nx, ny, nz, f0->r);
    free(u0);
    const double scale = bnorm > 0.0 ? bnorm : 1.0;

    or_residual(nx, ny, nz, x, y, z, u, b, f0->r);
    double rel = or_norm2_interior(nx, ny, nz, f0->r) / scale;
    if (hist) hist[0] = rel;
    int c = 0;
    st = OR_NOT_CONVERGED;
    if (tol > 0.0 && rel <= tol) st = OR_OK;
    while (st != OR_OK && c < max_cycles) {
        mg_cycle(&g, 0, c < n_f);
        c++;
        or_residual(nx, ny, nz, x, y, z, u, b, f0->r);
        rel = or_norm2_interior(nx, ny, nz, f0->r) / scale;
        if (hist) hist[c] = rel;
        if (!isfinite(rel)) { st = OR_NONFINITE; break; }
        if (tol > 0.0 && rel <= tol) st = OR_OK;
    }
    if (tol <= 0.0 && st == OR_NOT_CONVERGED) st = OR_OK;
    if (cycles_out) *cycles_out = c;
    for (int l = 0; l < L; l++) {
        level* v = &g.lv[l];
        for (int a = 0; a < 3; a++) free(v->c[a]);
        if (l > 0) { free(v->u); free(v->b); }
        free(v->r);
    }
    free(g.lu.LU); free(g.lu.piv);
    return st;
}

/* ------------------------------------------------------------------ projection */
/* Cell containing p: largest i with x[i] <= p, clamped to n-2 (a node hit uses the
 * cell to its right). */
static int find_cell(int n, const double* x, double p)
{
    int i = 0;
    while (i + 1 < n && x[i + 1] <= p) i++;
    if (i > n - 2) i = n - 2;
    return i;
}

/* Eq. 3.6: V_LM(R_i) = integral over the sphere surface of V y_LM.  Reading: the
 * measure is the unit-sphere solid angle, so that V = sum V_LM y_LM on the surface
 * (Eq. 3.5).  V comes from trilinear interpolation of the grid solution, as the
 * introduction's "interpolates onto the sphere boundaries". */
int or_project(int nx, int ny, int nz, const double* x, const double* y, const double* z,
               const double* u, int na, const double* pos, const double* R, int n_theta, int n_phi,
               double* vlm)
{
    double* t = malloc(sizeof(double) * n_theta);
    double* wt = malloc(sizeof(double) * n_theta);
    or_gauss_legendre(n_theta, t, wt);
    int st = OR_OK;
    for (int a = 0; a < na; a++) {
        double acc[25] = {0};
        for (int it = 0; it < n_theta; it++) {
            const double ct = t[it], stt = sqrt(1.0 - ct * ct);
            for (int ip = 0; ip < n_phi; ip++) {
                const double ph = 2.0 * PI * ip / n_phi;
                const double ux = stt * cos(ph), uy = stt * sin(ph), uz = ct;
                const double px = pos[3 * a] + R[a] * ux, py = pos[3 * a + 1] + R[a] * uy, pz = pos[3 * a + 2] + R[a] * uz;
                if (px < x[0] || px > x[nx - 1] || py < y[0] || py > y[ny - 1] || pz < z[0] || pz > z[nz - 1]) {
                    st = OR_GEOMETRY;
                    continue;
                }
                const int i = find_cell(nx, x, px), j = find_cell(ny, y, py), k = find_cell(nz, z, pz);
                const double tx = (px - x[i]) / (x[i + 1] - x[i]);
                const double ty = (py - y[j]) / (y[j + 1] - y[j]);
                const double tz = (pz - z[k]) / (z[k + 1] - z[k]);
                double V = 0.0;
                for (int c = 0; c < 2; c++)
                    for (int bb = 0; bb < 2; bb++)
                        for (int aa = 0; aa < 2; aa++)
                            V += (aa ? tx : 1.0 - tx) * (bb ? ty : 1.0 - ty) * (c ? tz : 1.0 - tz) *
                                 u[IDX(i + aa, j + bb, k + c, nx, ny)];
                double S[25];
                or_solid_harmonics(ux, uy, uz, S);
                const double wq = wt[it] * 2.0 * PI / n_phi;
                for (int lm = 0; lm < 25; lm++) acc[lm] += wq * V * S[lm];
            }
        }
        for (int lm = 0; lm < 25; lm++) vlm[25 * a + lm] = acc[lm];
    }
    free(t); free(wt);
    return st;
}

/* ------------------------------------------------------------------ whole step */
int or_poisson_solve(int na, const double* pos, const double* Z, const double* R, const double* w,
                     const double* zeta, const double* clm, const double* mesh, const int* ctl,
                     double tol, double* vlm, double* u, double* stats, double* hist)
{
    const int n = (int)mesh[0];
    const double c[3] = {mesh[1], mesh[2], mesh[3]};
    const double L = mesh[4], h_min = mesh[5], h_max = mesh[6], p_max = mesh[7];
    const int nu1 = ctl[0], nu2 = ctl[1], n_f = ctl[2], max_cycles = ctl[3], n_theta = ctl[4], n_phi = ctl[5];
    const int bc = ctl[6];   /* 0 multipole (default), 1 zero (Eq. 3.3), 2 exact superposition */
    if (stats) { stats[0] = 0; stats[1] = -1; stats[2] = OR_INVALID_ARG; }
    double* ax[3];
    for (int a = 0; a < 3; a++) {
        ax[a] = malloc(sizeof(double) * n);
        if (or_mesh_axis(n, c[a], L, h_min, h_max, p_max, ax[a], NULL) != OR_OK) {
            for (int b = 0; b <= a; b++) free(ax[b]);
            return OR_INVALID_ARG;
        }
    }
    /* geometry: spheres disjoint and at least two nodes inside the box faces */
    for (int i = 0; i < na; i++) {
        for (int a = 0; a < 3; a++)
            if (pos[3 * i + a] - R[i] < ax[a][2] || pos[3 * i + a] + R[i] > ax[a][n - 3]) {
                for (int b = 0; b < 3; b++) free(ax[b]);
                if (stats) stats[2] = OR_GEOMETRY;
                return OR_GEOMETRY;
            }
        for (int j = 0; j < i; j++) {
            const double dx = pos[3 * i] - pos[3 * j], dy = pos[3 * i + 1] - pos[3 * j + 1], dz = pos[3 * i + 2] - pos[3 * j + 2];
            if (sqrt(dx * dx + dy * dy + dz * dz) < R[i] + R[j]) {
                for (int b = 0; b < 3; b++) free(ax[b]);
                if (stats) stats[2] = OR_GEOMETRY;
                return OR_GEOMETRY;
            }
        }
    }
    const size_t N = (size_t)n * n * n;
    double* b = malloc(sizeof(double) * N);
    double* uu = u ? u : malloc(sizeof(double) * N);
    or_deposit(na, pos, Z, R, w, zeta, clm, n, n, n, ax[0], ax[1], ax[2], b, NULL);
    int st = OR_OK;
    for (size_t p = 0; p < N; p++)
        if (!isfinite(b[p])) { st = OR_NONFINITE; break; }
    int cycles = 0;
    if (st == OR_OK) {
        double Q[25];
        memset(uu, 0, sizeof(double) * N);
        if (bc == 0) {          /* multipole expansion of the grid charge, l <= 4 */
            or_multipoles(n, n, n, ax[0], ax[1], ax[2], b, c[0], c[1], c[2], Q);
            or_boundary_fill(n, n, n, ax[0], ax[1], ax[2], c[0], c[1], c[2], Q, uu);
        } else if (bc == 2) {   /* exact superposition of the atoms' potentials */
            or_boundary_exact(na, pos, Z, R, w, zeta, clm, n, n, n, ax[0], ax[1], ax[2], uu);
        }                       /* bc == 1: zero (Eq. 3.3) */
        st = or_mg_solve(n, n, n, ax[0], ax[1], ax[2], b, uu, nu1, nu2, n_f, tol, max_cycles, hist, &cycles);
        int sp = or_project(n, n, n, ax[0], ax[1], ax[2], uu, na, pos, R, n_theta, n_phi, vlm);
        if (st == OR_OK && sp != OR_OK) st = sp;
        if (stats) {
            stats[0] = cycles;
            stats[1] = hist ? hist[cycles] : -1.0;
        }
    }
    if (stats) stats[2] = st;
    free(b);
    if (!u) free(uu);
    for (int a = 0; a < 3; a++) free(ax[a]);
    return st;
}

/* ------------------------------------------------------------------ inside the spheres */
/* Logarithmic radial mesh of a sphere (the paper: "logarithmic, 429 points"; reading: the
 * last point on the sphere, the first at r_min):  r_j = R exp((j - (n-1)) dx),
 * dx = ln(R / r_min) / (n - 1). */
void or_radial_mesh(int n, double r_min, double R, double* r)
{
    const double dx = log(R / r_min) / (n - 1);
    for (int j = 0; j < n; j++) r[j] = R * exp((j - (n - 1)) * dx);
    r[n - 1] = R;
}

/* rho_LM(r_j) of atom a: Eq. 3.7's surface projection taken on the sphere of radius r_j about
 * the atom, sum_q w_q n_e(X_a + r_j u_q) y_LM(u_q), with the projection's n_theta-point
 * Gauss-Legendre x n_phi uniform rule.  out [na][25][n_rad]. */
int or_sphere_density(int na, const double* pos, const double* R, const double* w, const double* zeta,
                      const double* clm, int n_rad, double r_min, int n_theta, int n_phi, double* out)
{
    if (n_rad < 4 || !(r_min > 0.0)) return OR_INVALID_ARG;
    double* t = malloc(sizeof(double) * n_theta);
    double* wt = malloc(sizeof(double) * n_theta);
    or_gauss_legendre(n_theta, t, wt);
#pragma omp parallel for schedule(dynamic)
    for (int a = 0; a < na; a++) {
        double* rr = malloc(sizeof(double) * n_rad);
        or_radial_mesh(n_rad, r_min, R[a], rr);
        for (int j = 0; j < n_rad; j++) {
            double acc[25] = {0};
            for (int it = 0; it < n_theta; it++) {
                const double ct = t[it], stt = sqrt(1.0 - ct * ct);
                for (int ip = 0; ip < n_phi; ip++) {
                    const double ph = 2.0 * PI * ip / n_phi;
                    const double ux = stt * cos(ph), uy = stt * sin(ph), uz = ct;
                    const double rho = or_density(na, pos, R, w, zeta, clm, pos[3 * a] + rr[j] * ux,
                                                  pos[3 * a + 1] + rr[j] * uy, pos[3 * a + 2] + rr[j] * uz);
                    double S[25];
                    or_solid_harmonics(ux, uy, uz, S);
                    const double wq = wt[it] * 2.0 * PI / n_phi;
                    for (int lm = 0; lm < 25; lm++) acc[lm] += wq * rho * S[lm];
                }
            }
            for (int lm = 0; lm < 25; lm++) out[((size_t)a * 25 + lm) * n_rad + j] = acc[lm];
        }
        free(rr);
    }
    free(t); free(wt);
    return OR_OK;
}

/* integral of g over [x_j, x_{j+1}] on a uniform grid (step h, n >= 4 points): the cubic
 * through the four nearest samples */
static double seg_integral(const double* g, int n, int j, double h)
{
    if (j == 0) return h / 24.0 * (9.0 * g[0] + 19.0 * g[1] - 5.0 * g[2] + g[3]);
    if (j == n - 2) return h / 24.0 * (g[n - 4] - 5.0 * g[n - 3] + 19.0 * g[n - 2] + 9.0 * g[n - 1]);
    return h / 24.0 * (-g[j - 1] + 13.0 * g[j] + 13.0 * g[j + 1] - g[j + 2]);
}

/* Inner Dirichlet problem of sphere a (Eq. 3.4 with the boundary values of Eq. 3.6), in the
 * Green's-function form of Eq. 3.5:
 *   V_LM(r) = V_LM(R) (r/R)^L
 *           - 4pi/(2L+1) [ r^-(L+1) int_0^r rho_LM r'^(L+2) dr' + r^L int_r^R rho_LM r'^(1-L) dr'
 *                          - r^L R^-(2L+1) int_0^R rho_LM r'^(L+2) dr' ]
 *           + delta_L0 sqrt(4pi) Z (1/r - 1/R),
 * which solves (d2/dr2 + (2/r) d/dr - L(L+1)/r^2) V_LM = 4pi (rho_LM - delta_L0 Z delta) with
 * V_LM(R) given (reading of Eq. 3.5: its printed integrands are rho r^(L+2) and rho r^(1-L),
 * and its overall sign is the one that satisfies Eq. 3.4).  Integrals in x = ln r
 * (dr = r dx) with the cubic rule; on [0, r_0] rho is taken constant.  rho_lm, v: [na][25][n_rad];
 * v_R: [na][25]. */
int or_inner_solve(int na, const double* R, const double* Z, int n_rad, double r_min, const double* rho_lm,
                   const double* v_R, double* v)
{
    if (n_rad < 4 || !(r_min > 0.0)) return OR_INVALID_ARG;
    double* r = malloc(sizeof(double) * n_rad);
    double* g1 = malloc(sizeof(double) * n_rad);
    double* g2 = malloc(sizeof(double) * n_rad);
    double* I1 = malloc(sizeof(double) * n_rad);
    double* I2 = malloc(sizeof(double) * n_rad);
    for (int a = 0; a < na; a++) {
        or_radial_mesh(n_rad, r_min, R[a], r);
        const double h = log(R[a] / r_min) / (n_rad - 1);
        for (int lm = 0; lm < 25; lm++) {
            const int L = l_of(lm);
            const double* rho = rho_lm + ((size_t)a * 25 + lm) * n_rad;
            for (int j = 0; j < n_rad; j++) {
                g1[j] = rho[j] * pow(r[j], L + 2) * r[j];
                g2[j] = rho[j] * pow(r[j], 1 - L) * r[j];
            }
            I1[0] = rho[0] * pow(r[0], L + 3) / (L + 3);
            for (int j = 0; j + 1 < n_rad; j++) I1[j + 1] = I1[j] + seg_integral(g1, n_rad, j, h);
            I2[n_rad - 1] = 0.0;
            for (int j = n_rad - 2; j >= 0; j--) I2[j] = I2[j + 1] + seg_integral(g2, n_rad, j, h);
            const double Ra = R[a], vr = v_R[25 * a + lm];
            for (int j = 0; j < n_rad; j++) {
                const double x = r[j] / Ra, rl = pow(r[j], L);
                double val = vr * pow(x, L) - 4.0 * PI / (2 * L + 1) *
                                                  (I1[j] / pow(r[j], L + 1) + rl * I2[j] -
                                                   rl * I1[n_rad - 1] / pow(Ra, 2 * L + 1));
                if (L == 0) val += sqrt(4.0 * PI) * Z[a] * (1.0 / r[j] - 1.0 / Ra);
                v[((size_t)a * 25 + lm) * n_rad + j] = val;
            }
        }
    }
    free(r); free(g1); free(g2); free(I1); free(I2);
    return OR_OK;
}

/* ------------------------------------------------------------------ raw density (Eq. 3.1) */
/* rho_00 at radius r from its samples on the logarithmic mesh: cubic Lagrange interpolation
 * in x = ln r on the four nearest samples; below r_min the straight line through the first
 * two samples (the density has a cusp at the nucleus: constant would miss -zeta rho r_min) */
static double radial_interp(const double* f, int n, double r_min, double dx, double r)
{
    if (r <= r_min) {
        const double r1 = r_min * exp(dx);
        return f[0] + (f[1] - f[0]) * (r - r_min) / (r1 - r_min);
    }
    const double t = log(r / r_min) / dx;
    int j = (int)floor(t);
    if (j < 1) j = 1;
    if (j > n - 3) j = n - 3;
    const double s = t - j;   /* position relative to sample j; the stencil is j-1 .. j+2 */
    const double l0 = -s * (s - 1.0) * (s - 2.0) / 6.0, l1 = (s + 1.0) * (s - 1.0) * (s - 2.0) / 2.0;
    const double l2 = -(s + 1.0) * s * (s - 2.0) / 2.0, l3 = (s + 1.0) * s * (s - 1.0) / 6.0;
    return l0 * f[j - 1] + l1 * f[j] + l2 * f[j + 1] + l3 * f[j + 2];
}

/* Pseudo-density of each sphere from the density's own spherical component (Section 3's
 * three constraints, as or_sphere_params but with rho taken from the radial table):
 * q = sqrt(4pi) int_0^R rho_00 r^2 dr - Z (cubic rule in ln r, rho_00 constant on [0, r_min]),
 * rho(R) = rho_00(R)/sqrt(4pi), rho'(R) = (d rho_00/d ln r)(R) / (R sqrt(4pi)) with the
 * one-sided fourth-order difference; coef = (a, b, c) of a + b r^2 + c r^4. */
int or_raw_sphere_params(int na, const double* Z, const double* R, int n_rad, double r_min, const double* rho00,
                         double* q, double* rhoR, double* drhoR, double* coef)
{
    if (n_rad < 5 || !(r_min > 0.0)) return OR_INVALID_ARG;
    double* g = malloc(sizeof(double) * n_rad);
    double* r = malloc(sizeof(double) * n_rad);
    const double s4 = sqrt(4.0 * PI);
    for (int i = 0; i < na; i++) {
        const double* f = rho00 + (size_t)i * n_rad;
        or_radial_mesh(n_rad, r_min, R[i], r);
        const double h = log(R[i] / r_min) / (n_rad - 1);
        for (int j = 0; j < n_rad; j++) g[j] = f[j] * r[j] * r[j] * r[j];
        double acc = f[0] * r[0] * r[0] * r[0] / 3.0;
        for (int j = 0; j + 1 < n_rad; j++) acc += seg_integral(g, n_rad, j, h);
        q[i] = s4 * acc - Z[i];
        const int m = n_rad - 1;
        rhoR[i] = f[m] / s4;
        drhoR[i] = (25.0 * f[m] - 48.0 * f[m - 1] + 36.0 * f[m - 2] - 16.0 * f[m - 3] + 3.0 * f[m - 4]) /
                   (12.0 * h) / (R[i] * s4);
        const double Ri = R[i];
        double M[3][3] = {{4.0 * PI * pow(Ri, 3) / 3.0, 4.0 * PI * pow(Ri, 5) / 5.0, 4.0 * PI * pow(Ri, 7) / 7.0},
                          {1.0, Ri * Ri, pow(Ri, 4)},
                          {0.0, 2.0 * Ri, 4.0 * pow(Ri, 3)}};
        double rhs[3] = {q[i], rhoR[i], drhoR[i]};
        solve3(M, rhs, &coef[3 * i]);
    }
    free(g); free(r);
    return OR_OK;
}

/* Deposit from a raw density: b = 4pi rho~_grid with rho~_grid = ne outside the spheres and
 * ne - rho_00(r)/sqrt(4pi) + pseudo(r) inside sphere i (the monopole swap of Section 1 with the
 * spherical part from the radial table).  ne: [nz][ny][nx]; rho00: [na][n_rad]. */
int or_raw_deposit(int na, const double* pos, const double* Z, const double* R, int nx, int ny, int nz,
                   const double* x, const double* y, const double* z, const double* ne, int n_rad, double r_min,
                   const double* rho00, double* b, int* owner)
{
    double* q = malloc(sizeof(double) * na);
    double* rhoR = malloc(sizeof(double) * na);
    double* drhoR = malloc(sizeof(double) * na);
    double* coef = malloc(sizeof(double) * 3 * na);
    const int st = or_raw_sphere_params(na, Z, R, n_rad, r_min, rho00, q, rhoR, drhoR, coef);
    if (st == OR_OK) {
        const double s4 = sqrt(4.0 * PI);
#pragma omp parallel for schedule(dynamic)
        for (int k = 0; k < nz; k++)
            for (int j = 0; j < ny; j++)
                for (int i = 0; i < nx; i++) {
                    int own = -1;
                    double r = 0.0;
                    for (int a = 0; a < na; a++) {
                        const double dx = x[i] - pos[3 * a], dy = y[j] - pos[3 * a + 1], dz = z[k] - pos[3 * a + 2];
                        const double ra = sqrt(dx * dx + dy * dy + dz * dz);
                        if (ra < R[a]) { own = a; r = ra; break; }
                    }
                    const size_t P = IDX(i, j, k, nx, ny);
                    double val = ne[P];
                    if (own >= 0) {
                        const double hh = log(R[own] / r_min) / (n_rad - 1);
                        const double rho0 = radial_interp(rho00 + (size_t)own * n_rad, n_rad, r_min, hh, r) / s4;
                        const double* c = &coef[3 * own];
                        val = val - rho0 + (c[0] + c[1] * r * r + c[2] * r * r * r * r);
                    }
                    b[P] = 4.0 * PI * val;
                    if (owner) owner[P] = own;
                }
    }
    free(q); free(rhoR); free(drhoR); free(coef);
    return st;
}

/* ------------------------------------------------------------------ interstitial H and S (Eq. 3.11-3.14) */
/* Interstitial overlap and Hamiltonian contributions of a Slater-type basis (Eq. 3.13:
 * phi_inlm = r_i^(n-1) e^{-zeta r_i} y_lm(r^_i), for every atom i and every (n, l, zeta) of the
 * basis table, all m), summed over the grid nodes outside every sphere with the dual-cell
 * volume (the grid-point form S^1, H^1 of Section 3):
 *   S_ab = sum_P phi_a(P) phi_b(P) Vol(P),
 *   H_ab = 1/2 sum_P (phi_a(P) phit_b(P) + phi_b(P) phit_a(P)) Vol(P),
 *   phit = 1/2 [(l(l+1) - n(n-1)) r^(n-3) + 2 zeta n r^(n-2) - zeta^2 r^(n-1)] e^{-zeta r} y_lm
 *          + V(P) phi (Eq. 3.14, -1/2 Lap + V applied to phi).
 * Function order: atom-major, then the basis table's order, then m = -l..l (lm = l^2+l+m).
 * V: potential energy at the nodes [nz][ny][nx]; S, H: [M][M], M = na * sum(2l+1). */
int or_interstitial_hs(int na, const double* pos, const double* R, int nb, const int* bn, const int* bl,
                       const double* bz, int nx, int ny, int nz, const double* x, const double* y, const double* z,
                       const double* V, double* S, double* H)
{
    int per = 0;
    for (int q = 0; q < nb; q++) {
        if (bl[q] < 0 || bl[q] > 4 || bn[q] < bl[q] + 1) return OR_INVALID_ARG;
        per += 2 * bl[q] + 1;
    }
    const int M = na * per;
    double *vx = malloc(sizeof(double) * nx), *vy = malloc(sizeof(double) * ny), *vz = malloc(sizeof(double) * nz);
    or_dual_lengths(nx, x, vx);
    or_dual_lengths(ny, y, vy);
    or_dual_lengths(nz, z, vz);
    memset(S, 0, sizeof(double) * M * M);
    memset(H, 0, sizeof(double) * M * M);
    const int nthr = omp_get_max_threads();
    double* part = calloc((size_t)nthr * 2 * M * M, sizeof(double));
#pragma omp parallel
    {
        double* ph = malloc(sizeof(double) * M);
        double* pt = malloc(sizeof(double) * M);
        double* Sp = part + (size_t)omp_get_thread_num() * 2 * M * M;
        double* Hp = Sp + (size_t)M * M;
#pragma omp for schedule(static)
        for (int k = 0; k < nz; k++)
            for (int j = 0; j < ny; j++)
                for (int i = 0; i < nx; i++) {
                    int inside = 0;
                    for (int a = 0; a < na && !inside; a++) {
                        const double dx = x[i] - pos[3 * a], dy = y[j] - pos[3 * a + 1], dz = z[k] - pos[3 * a + 2];
                        if (sqrt(dx * dx + dy * dy + dz * dz) < R[a]) inside = 1;
                    }
                    if (inside) continue;
                    const double vol = vx[i] * vy[j] * vz[k], Vp = V[IDX(i, j, k, nx, ny)];
                    int f = 0;
                    for (int a = 0; a < na; a++) {
                        const double dx = x[i] - pos[3 * a], dy = y[j] - pos[3 * a + 1], dz = z[k] - pos[3 * a + 2];
                        const double r = sqrt(dx * dx + dy * dy + dz * dz);
                        double Sl[25];
                        or_solid_harmonics(dx, dy, dz, Sl);
                        for (int q = 0; q < nb; q++) {
                            const int n = bn[q], l = bl[q];
                            const double zt = bz[q], e = exp(-zt * r);
                            const double rad = pow(r, n - 1 - l) * e;   /* r^(n-1) y_lm = r^(n-1-l) S_lm */
                            const double kin = 0.5 * ((l * (l + 1) - n * (n - 1)) / (r * r) + 2.0 * zt * n / r - zt * zt) * rad;
                            for (int m = -l; m <= l; m++) {
                                const double s = Sl[l * l + l + m];
                                ph[f] = rad * s;
                                pt[f] = kin * s + Vp * rad * s;
                                f++;
                            }
                        }
                    }
                    for (int p = 0; p < M; p++) {
                        const double wp = vol * ph[p], wt = vol * pt[p];
                        for (int qq = 0; qq < M; qq++) {
                            Sp[(size_t)p * M + qq] += wp * ph[qq];
                            Hp[(size_t)p * M + qq] += 0.5 * (wp * pt[qq] + wt * ph[qq]);
                        }
                    }
                }
        free(ph); free(pt);
    }
    for (int t = 0; t < nthr; t++)
        for (size_t e = 0; e < (size_t)M * M; e++) {
            S[e] += part[(size_t)t * 2 * M * M + e];
            H[e] += part[(size_t)t * 2 * M * M + (size_t)M * M + e];
        }
    free(part); free(vx); free(vy); free(vz);
    return OR_OK;
}
