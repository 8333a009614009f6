/*
 * lasto_oracle.h -- plain FP64 CPU oracle of the LASTO interstitial Poisson step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA library, and the CUDA library never
 * calls it.
 *
 * Each routine is written step by step from the paper (Kang, Davenport, Glimm,
 * Keyes, McGuigan, "Linear Augmented Slater-Type Orbital Method for Free
 * Standing Clusters"), Sections 2-3, with the readings listed beside each
 * function where the paper is silent or garbled.  Everything is FP64 and
 * unblocked; the only parallelism is an OpenMP split of independent node loops,
 * and every reduction is summed in a fixed order so results do not depend on
 * the thread count.
 *
 * Conventions
 *   Grids are vertex-centred tensor-product meshes with nx*ny*nz nodes stored
 *   x-fastest: index = (k*ny + j)*nx + i.  Nodes on the outer faces carry
 *   Dirichlet values.  Atom arrays: pos[n][3], Z[n], R[n], w[n][3], zeta[n][3],
 *   c_lm[n][24] (l = 1..4, slot l*l+l+m-1).  Real spherical harmonics are the
 *   orthonormal ones without the Condon-Shortley phase; lm = l*l + l + m.
 *   Sign (Eq. 2.6 / 3.2): the solver finds u with Lap u = 4*pi*rho_tilde, where
 *   rho_tilde is the electron-sign pseudo-density, so u is the electrostatic
 *   potential (u -> +Z/r near a bare nucleus).
 */
#ifndef LASTO_ORACLE_H
#define LASTO_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_OK = 0, OR_INVALID_ARG = 1, OR_GEOMETRY = 2, OR_NONFINITE = 3, OR_NOT_CONVERGED = 4 };

/* Real solid harmonics S_lm(x) = r^l y_lm(x/r), l <= 4, 25 values (Eq. 3.1's y_LM). */
void or_solid_harmonics(double x, double y, double z, double* S);

/* n-point Gauss-Legendre rule on [-1, 1], ascending nodes. */
int or_gauss_legendre(int n, double* t, double* w);

/* One mesh axis (Section 3: fine near the atoms, coarse far away; Dirichlet at the
 * edge).  x(xi) = c + A xi + B sign(xi)|xi|^p, xi = (i-m)/m, m = (n-1)/2, with
 * A = h_min m, A + B = L and end slope A + p B = h_max m; if p > p_max then p = p_max
 * and A, B follow from the other two conditions.  info = {A, B, p, h_centre, h_edge}. */
int or_mesh_axis(int n, double c, double L, double h_min, double h_max, double p_max, double* x, double* info);

/* Dual-cell lengths: (x[i+1]-x[i-1])/2 inside, half a spacing at the two ends. */
void or_dual_lengths(int n, const double* x, double* v);

/* True electron density n_e at a point (stands in for Eq. 3.15's density). */
double or_density(int na, const double* pos, const double* R, const double* w, const double* zeta,
                  const double* clm, double x, double y, double z);
void or_density_grid(int na, const double* pos, const double* R, const double* w, const double* zeta,
                     const double* clm, int nx, int ny, int nz, const double* x, const double* y,
                     const double* z, double* out);

/* Spherical (monopole) part of n_e about atom i at radius r, and its r-derivative. */
void or_monopole(int na, const double* pos, const double* w, const double* zeta, int i, double r,
                 double* rho0, double* drho0);

/* Pseudo-density of each sphere (Section 3, constraints beside Eq. 3.2-3.3):
 * q[i] = 4 pi int_0^R rho0 r^2 dr - Z, rhoR, drhoR = rho0(R), rho0'(R), and
 * coef[i] = (a, b, c) of rho_tilde(r) = a + b r^2 + c r^4. */
void or_sphere_params(int na, const double* pos, const double* Z, const double* R, const double* w,
                      const double* zeta, double* q, double* rhoR, double* drhoR, double* coef);

/* Right-hand side b = 4 pi rho_tilde_grid at every node (Section 1 last paragraphs and
 * Section 3): inside sphere i the monopole of n_e is swapped for rho_tilde_i, every
 * other part of n_e stays on the grid.  owner[node] = sphere index or -1 (may be NULL). */
int or_deposit(int na, const double* pos, const double* Z, const double* R, const double* w,
               const double* zeta, const double* clm, int nx, int ny, int nz, const double* x,
               const double* y, const double* z, double* b, int* owner);

/* Q_lm = sum_nodes (b/4pi) vol S_lm(node - centre), l <= 4. */
void or_multipoles(int nx, int ny, int nz, const double* x, const double* y, const double* z,
                   const double* b, double cx, double cy, double cz, double* Q);

/* Dirichlet face values u = -sum_lm 4pi/(2l+1) Q_lm y_lm / r^(l+1) (Eq. 2.7). */
void or_boundary_fill(int nx, int ny, int nz, const double* x, const double* y, const double* z,
                      double cx, double cy, double cz, const double* Q, double* u);

/* Finite-difference Laplacian on the graded mesh, interior nodes; boundary entries of
 * Au / r are set to zero. */
void or_apply_A(int nx, int ny, int nz, const double* x, const double* y, const double* z,
                const double* u, double* Au);
void or_residual(int nx, int ny, int nz, const double* x, const double* y, const double* z,
                 const double* u, const double* b, double* r);
double or_norm2_interior(int nx, int ny, int nz, const double* r);

/* One red (colour 0: i+j+k even) or black (colour 1) Gauss-Seidel half sweep. */
void or_rbgs_half(int nx, int ny, int nz, const double* x, const double* y, const double* z,
                  double* u, const double* b, int colour);

/* Full weighting bc = Vc^-1 P^T Vf r onto the every-other-node coarse mesh. */
void or_restrict(int nx, int ny, int nz, const double* x, const double* y, const double* z,
                 const double* r, double* bc);
/* u += P ec, P = trilinear interpolation in physical coordinates. */
void or_prolong_add(int nx, int ny, int nz, const double* x, const double* y, const double* z,
                    const double* ec, double* u);

/* Exact solve of A e = b on the interior with zero boundary values (dense LU, partial pivoting). */
int or_coarse_solve(int nx, int ny, int nz, const double* x, const double* y, const double* z,
                    const double* b, double* e);

/* Number of multigrid levels for n nodes per axis (coarsen while any axis has > 9 nodes). */
int or_num_levels(int nx, int ny, int nz);

/* Multigrid on A u = b (Section 3, "finite difference scheme and a multigrid method").
 * u holds the Dirichlet values on its faces and the initial interior guess.  Runs n_f
 * F-cycles, then V(nu1,nu2)-cycles until ||b - A u|| <= tol ||b_eff|| or max_cycles
 * cycles in all; hist[c] = relative residual after cycle c (hist[0] = start).
 * With tol <= 0 exactly max_cycles cycles run.  Returns OR_OK or OR_NOT_CONVERGED. */
int or_mg_solve(int nx, int ny, int nz, const double* x, const double* y, const double* z,
                const double* b, double* u, int nu1, int nu2, int n_f, double tol, int max_cycles,
                double* hist, int* cycles_out);

/* V_LM(R_i) = int y_LM V dOmega on each sphere surface (Eq. 3.6), Gauss-Legendre in
 * cos(theta) x uniform phi, V from trilinear interpolation of u. vlm[na][25]. */
int or_project(int nx, int ny, int nz, const double* x, const double* y, const double* z,
               const double* u, int na, const double* pos, const double* R, int n_theta, int n_phi,
               double* vlm);

/* The whole step: mesh, deposit, multipoles, faces, multigrid, projection.
 * mesh = {n, cx, cy, cz, L, h_min, h_max, p_max} (cubic box), ctl = {nu1, nu2, n_f,
 * max_cycles, n_theta, n_phi}, tol.  Outputs: vlm[na][25]; u[n^3] (may be NULL);
 * stats = {cycles, rel_resid, status, Q_00.., } (stats[0..2]); hist[max_cycles+1]. */
int or_poisson_solve(int na, const double* pos, const double* Z, const double* R, const double* w,
                     const double* zeta, const double* clm, const double* mesh, const int* ctl,
                     double tol, double* vlm, double* u, double* stats, double* hist);

/* Exact superposition Dirichlet values: on the six faces, the continuum potential of every
 * atom (normalised-exponential shells, nucleus, exterior multipoles of the nonspherical part). */
void or_boundary_exact(int na, const double* pos, const double* Z, const double* R, const double* w,
                       const double* zeta, const double* clm, int nx, int ny, int nz, const double* x,
                       const double* y, const double* z, double* u);

/* Inside the spheres (Section 3, Eq. 3.4-3.7).  Radial mesh r_j = R exp((j-(n-1)) dx),
 * dx = ln(R/r_min)/(n-1); rho_LM(r_j) by the surface projection of Eq. 3.7 at each radius;
 * the inner Dirichlet solve of Eq. 3.4 in the Green's-function form of Eq. 3.5. */
void or_radial_mesh(int n, double r_min, double R, double* r);
int or_sphere_density(int na, const double* pos, const double* R, const double* w, const double* zeta,
                      const double* clm, int n_rad, double r_min, int n_theta, int n_phi, double* out);
int or_inner_solve(int na, const double* R, const double* Z, int n_rad, double r_min, const double* rho_lm,
                   const double* v_R, double* v);

/* Raw density (Eq. 3.1's representation: a grid density and, per sphere, the spherical
 * component rho_00 on the logarithmic radial mesh): pseudo-density from the table and the
 * deposit with the monopole swap. */
int or_raw_sphere_params(int na, const double* Z, const double* R, int n_rad, double r_min, const double* rho00,
                         double* q, double* rhoR, double* drhoR, double* coef);
int or_raw_deposit(int na, const double* pos, const double* Z, const double* R, int nx, int ny, int nz,
                   const double* x, const double* y, const double* z, const double* ne, int n_rad, double r_min,
                   const double* rho00, double* b, int* owner);

/* Interstitial overlap and Hamiltonian contributions of a Slater-type basis (Eq. 3.11-3.14,
 * grid-point form): nodes outside every sphere, dual-cell volumes; bn, bl, bz: the basis
 * table's n, l, zeta (nb entries); V: potential energy at the nodes; S, H: [M][M],
 * M = na * sum(2l+1), functions atom-major, table order, m = -l..l. */
int or_interstitial_hs(int na, const double* pos, const double* R, int nb, const int* bn, const int* bl,
                       const double* bz, int nx, int ny, int nz, const double* x, const double* y, const double* z,
                       const double* V, double* S, double* H);

#ifdef __cplusplus
}
#endif
#endif
