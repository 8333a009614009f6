/*
 * lasto_poisson.h -- C ABI of the GB300 (sm_103a) LASTO interstitial Poisson step.
 *
 * The step is the Poisson solve between the atom spheres of a free-standing
 * cluster in the Linear Augmented Slater-Type Orbital method (Kang, Davenport,
 * Glimm, Keyes, McGuigan; Section 3, Eq. 3.2-3.6, with Section 1's description
 * of the pseudo-density):
 *   1. inside every sphere the monopole of the electron density is replaced by a
 *      smooth pseudo-density with the same charge (nucleus included) and the same
 *      value and slope at the sphere radius; the nonspherical terms stay on the
 *      grid as they are;
 *   2. the pseudo-density is deposited on a graded tensor-product mesh and the
 *      box faces get Dirichlet values from the cluster's multipole expansion;
 *   3. multigrid (7-point finite differences, red-black Gauss-Seidel, full
 *      weighting, trilinear prolongation, exact coarse solve), accelerated by
 *      conjugate gradients, solves Lap u = 4 pi rho_tilde between the spheres;
 *   4. the potential is interpolated onto every sphere surface and projected on
 *      real spherical harmonics up to l = 4 (Eq. 3.6), the boundary data of the
 *      inner Dirichlet problem (Eq. 3.4-3.5).
 *
 * Conventions used by every entry point
 *   - Units: bohr and hartree.  u is the electrostatic potential: Lap u =
 *     4 pi rho_tilde with rho_tilde the electron-sign pseudo-density, so
 *     u -> +Z/r near a bare nucleus (the sign of Eq. 2.6).
 *   - Grids: n[0]*n[1]*n[2] nodes, x-fastest, index (k*n[1] + j)*n[0] + i, FP64.
 *     Nodes on the six faces carry Dirichlet values.  n[a] is odd and coarsens
 *     (n+1)/2 repeatedly to at most 9 nodes per axis; a grid holds fewer than 2^31
 *     nodes (the kernels index with 31 bits; larger grids are INVALID_ARG).
 *   - Atoms: pos[n_atoms][3], Z[n_atoms], R[n_atoms], slater_w[n_atoms][3]
 *     (electrons in each normalised Slater term zeta^3/(8 pi) e^{-zeta r}),
 *     slater_zeta[n_atoms][3] (the same three exponents for every atom of a
 *     cluster), c_lm[n_atoms][24] (coefficient of (r/R)^l y_lm in the
 *     nonspherical part, l = 1..4, slot l*l + l + m - 1).
 *   - Real spherical harmonics: orthonormal, no Condon-Shortley phase,
 *     lm = l*l + l + m, m > 0 ~ cos(m phi), m < 0 ~ sin(|m| phi).
 *   - Every pointer argument is DEVICE memory unless it says "host".  The caller
 *     owns all inputs and outputs and the stream; nothing is freed or retained
 *     beyond the call except inside a handle.
 *   - Every call is asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *     default stream).  Device-detected outcomes are written to device or host
 *     status memory as stated and are valid after the stream synchronises.
 *   - Return value: LASTO_OK or an error code for what the host can detect
 *     (bad arguments, CUDA launch errors).  No exception or abort crosses the ABI.
 */
#ifndef LASTO_POISSON_H
#define LASTO_POISSON_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum lasto_status {
    LASTO_OK = 0,
    LASTO_ERR_INVALID_ARG = 1,   /* bad sizes, null pointers, mesh that cannot coarsen, non-uniform zeta */
    LASTO_ERR_GEOMETRY = 2,      /* spheres overlap, or a sphere is not two nodes inside the box */
    LASTO_ERR_NONFINITE = 3,     /* NaN/Inf in the deposited density or in the iteration */
    LASTO_ERR_NOT_CONVERGED = 4, /* cycle cap reached; outputs are written and stats hold the residual */
    LASTO_ERR_TIMEOUT = 5,       /* a bounded device wait ran out */
    LASTO_ERR_CUDA = 6,          /* a CUDA call failed; lasto_poisson_last_error() has the text */
    LASTO_ERR_NO_MEMORY = 7      /* a solve needs more than the handle's workspace */
};

enum lasto_precision {
    LASTO_PREC_FP64 = 0,  /* everything in FP64 ("plain" form) */
    LASTO_PREC_MIXED = 1  /* defect correction: FP64 residual and correction accumulation around
                             an FP32 multigrid-preconditioned CG (FP32 smoothing, restriction,
                             prolongation and CG vectors); the density exponentials in FP32-pair
                             arithmetic (about 44 bits); moments and projection stay FP64 */
};

enum lasto_cycle {
    LASTO_CYCLE_V = 0,    /* stationary V(nu1,nu2)-cycles from the start */
    LASTO_CYCLE_FV = 1,   /* one F-cycle, then V-cycles */
    LASTO_CYCLE_PCG = 2   /* conjugate gradients preconditioned by one symmetric V-cycle (default) */
};

/* Dirichlet values on the box faces.  MULTIPOLE: the l <= 4 exterior expansion of the grid
 * charge about the box centre (Eq. 2.7's decay made finite; default).  ZERO: V_C = 0 as
 * Eq. 3.3 states.  EXACT: the superposition of every atom's continuum potential (nucleus,
 * normalised Slater shells Z/r - sum_k w_k [1/r - e^{-zeta_k r}(1/r + zeta_k/2)], exterior
 * multipoles of the nonspherical part), exact for the density model outside the spheres. */
enum lasto_boundary {
    LASTO_BC_MULTIPOLE = 0,
    LASTO_BC_ZERO = 1,
    LASTO_BC_EXACT = 2
};

typedef struct lasto_config {
    int n_max;        /* largest nodes per axis any solve will use (sizes the workspace) */
    int max_atoms;    /* largest total atom count per solve call */
    int max_batch;    /* largest number of clusters per solve call */
    int precision;    /* enum lasto_precision */
    int cycle;        /* enum lasto_cycle */
    int nu1, nu2;     /* pre/post Gauss-Seidel sweeps per level (red+black = one sweep; the mixed
                         precision's one-block coarse levels use nu_coarse) */
    int max_cycles;   /* cap on cycles / CG iterations */
    double rel_tol;   /* stop when ||b - A u||_2 <= rel_tol ||b_eff||_2 (b_eff: b with the faces moved in) */
    int n_theta;      /* Gauss-Legendre points in cos(theta) of the sphere quadrature (<= 32) */
    int n_phi;        /* uniform points in phi (<= 64) */
    int launch;       /* 0: one CUDA graph per solve, iteration loop on the device (default;
                         each cluster of a batch an independent branch of the graph);
                         1: the same kernels launched directly with a host-side loop that
                         synchronises once per iteration (for profilers that cannot see
                         kernels inside conditional graph nodes);
                         2: one CUDA graph in which the mixed-precision clusters of a batch
                         whose grids have the same shape run their iterations in lockstep:
                         every kernel of an iteration is launched once for all of them (a
                         cluster whose loop has ended returns at once), with the same
                         arithmetic per cluster as 0 (bitwise the same results) */
    int boundary;     /* enum lasto_boundary: Dirichlet values on the box faces */
    int nu_coarse;    /* pre/post sweeps per level on the coarse levels the FP32 cycle of the
                         mixed precision runs inside one thread block (at most 17 nodes per axis,
                         above the exact solve); >= 0.  The other levels use nu1/nu2. */
    int nu_fine;      /* pre/post sweeps on the finest level when > 0 (0: nu1/nu2 there too) */
} lasto_config;

/* Fills cfg with the defaults: n_max 129, max_atoms 561, max_batch 1, FP64, PCG,
 * multipole faces, nu1 = nu2 = 4 (the fastest time to 1e-10 measured on GB300 for both precisions: more sweeps
 * per level cost less than the CG iterations and reductions they save), nu_coarse = 4 (1 keeps
 * the Pd55 129^3 iteration count and shortens each cycle, but costs iterations on smaller
 * grids), nu_fine = 0, 50 cycles, rel_tol 1e-10, 16 x 32 sphere points, graph launch. */
void lasto_config_default(lasto_config* cfg);

typedef struct lasto_cluster {
    int n_atoms;
    const double* pos;          /* [n_atoms][3] device */
    const double* Z;            /* [n_atoms]    device */
    const double* R;            /* [n_atoms]    device */
    const double* slater_w;     /* [n_atoms][3] device */
    const double* slater_zeta;  /* [n_atoms][3] device */
    const double* c_lm;         /* [n_atoms][24] device */
    int n[3];                   /* nodes per axis */
    const double* x;            /* [n[0]] device node coordinates, strictly increasing */
    const double* y;            /* [n[1]] device */
    const double* z;            /* [n[2]] device */
    double centre[3];           /* host values: expansion centre of the boundary multipoles */
} lasto_cluster;

typedef struct lasto_stats {
    int cycles;         /* V-cycles or CG iterations run (all inner iterations for MIXED) */
    int status;         /* enum lasto_status of this cluster */
    double rel_resid;   /* final ||b - A u|| / ||b_eff|| (true residual, recomputed in FP64) */
    double bnorm;       /* ||b_eff|| */
    int outer;          /* FP64 defect-correction steps (MIXED with CG), else 0 */
    int guess;          /* 1: the solve started from the learned guess (lasto_poisson_set_guess) */
} lasto_stats;

typedef struct lasto_poisson lasto_poisson;   /* opaque; owns workspace, plans and CUDA graphs */

/* Smoother tuning (no counterpart in the paper, which gives no implementation).  The first
 * solve of each new batch layout times, per level shape and precision, the red-black
 * smoother as in-place half sweeps (128, 256 or 512 threads per block over the flat node
 * index, or one block per (j, k) row: threads = 0) and as fused passes of the z-slab and
 * register-column kernels (several tile shapes), and the cycle uses the fastest; all give
 * bitwise the same iterates.  lasto_poisson_tune_table writes the table as
 * text, one line per shape: "nx ny nz elem_bytes fused threads tx ty kz sweeps_per_pass us"
 * (NUL-terminated into buf when cap > 0) and returns its length, -1 for a null handle.
 * lasto_poisson_set_tune_table adds such lines (shapes it lists are then not timed);
 * INVALID_ARG for a malformed line or an unusable choice (the fused passes of the pre- and
 * post-smoothing must together be even in number). */
int lasto_poisson_tune_table(const lasto_poisson* h, char* buf, size_t cap);
int lasto_poisson_set_tune_table(lasto_poisson* h, const char* text);

/* Raw density (Eq. 3.1's representation: the density on the grid and, inside each sphere,
 * its spherical-harmonic components on the logarithmic radial mesh; the entry point for
 * densities that do not come from the synthetic Slater model, e.g. an SCF iteration's).
 * density: the electron density at every node (device [n2][n1][n0], x fastest, the same
 * nodes as x, y, z); rho00: each sphere's spherical component rho_00(r_j) = integral of the
 * density times y_00 over the sphere of radius r_j (device [n_atoms][n_rad]) on the mesh
 * r_j = R_a exp((j - (n_rad-1)) dx), dx = ln(R_a/r_min)/(n_rad-1).  From each table: q =
 * sqrt(4pi) int_0^R rho_00 r^2 dr - Z (cubic rule in ln r), rho(R), rho'(R) (one-sided
 * fourth-order difference in ln r) and the quartic pseudo-density of Section 3; inside the
 * sphere the deposit takes density - rho_00(r)/sqrt(4pi) + pseudo(r) with rho_00(r) by cubic
 * interpolation in ln r (the straight line through the first two samples below r_min).  The
 * rest of the solve is lasto_poisson_solve's (faces: multipole or zero; EXACT needs the model
 * density and gives INVALID_ARG).  Arguments otherwise as lasto_poisson_solve; n_rad >= 5. */
typedef struct lasto_raw_cluster {
    int n_atoms;
    const double* pos;      /* [n_atoms][3] device */
    const double* Z;        /* [n_atoms] device */
    const double* R;        /* [n_atoms] device */
    int n[3];
    const double* x;        /* [n[0]] device node coordinates */
    const double* y;
    const double* z;
    double centre[3];       /* host: expansion centre of the boundary multipoles */
    const double* density;  /* [n[2]][n[1]][n[0]] device */
    int n_rad;
    double r_min;
    const double* rho00;    /* [n_atoms][n_rad] device */
} lasto_raw_cluster;
int lasto_poisson_solve_raw(lasto_poisson* h, const lasto_raw_cluster* clusters, int n_clusters, double* v_lm,
                            double* potential, const double* guess, lasto_stats* stats, void* stream);
/* The raw deposit alone: b (device [N]) = 4 pi rho~_grid, owner (optional, device int [N]) the
 * sphere holding each node or -1, status (device int) GEOMETRY / NONFINITE. */
int lasto_op_raw_deposit(const lasto_raw_cluster* cl, double* b, int* owner, int* status, void* stream);

/* Inside the atom spheres (Section 3, Eq. 3.4-3.7).  Radial mesh of sphere a (the paper:
 * logarithmic, 429 points): r_j = R_a exp((j - (n_rad-1)) dx), dx = ln(R_a / r_min)/(n_rad-1),
 * so r_0 = r_min and r_{n_rad-1} = R_a.
 *
 * lasto_op_sphere_density: rho_LM(r_j), the surface projection of Eq. 3.7 on the sphere of
 * radius r_j about each atom (n_theta-point Gauss-Legendre in cos(theta) x n_phi uniform
 * phi), of the cluster's electron density (all atoms' Slater shells plus the atom's own
 * nonspherical part).  rho_lm: device [n_atoms][25][n_rad]; the cluster's arrays and axes
 * are device arrays as for lasto_poisson_solve (the axes are used for the sphere geometry
 * check, whose failure sets *status = LASTO_ERR_GEOMETRY).
 *
 * lasto_op_inner_solve: the inner Dirichlet problem of Eq. 3.4 with the boundary values
 * V_LM(R) of Eq. 3.6 (v_R: device [n_atoms][25], as written by lasto_poisson_solve), solved
 * in the Green's-function form of Eq. 3.5 (read with the overall sign that satisfies Eq. 3.4,
 * and integrands rho r^(L+2), rho r^(1-L)):
 *   V_LM(r) = V_LM(R)(r/R)^L - 4pi/(2L+1)[r^-(L+1) I1(r) + r^L I2(r) - r^L R^-(2L+1) I1(R)]
 *             + delta_L0 sqrt(4pi) Z (1/r - 1/R),
 * I1(r) = int_0^r rho_LM r'^(L+2) dr', I2(r) = int_r^R rho_LM r'^(1-L) dr', integrated in
 * ln r (cubic through the four nearest samples per interval; rho constant on [0, r_min]).
 * R, Z: device [n_atoms]; rho_lm, v: device [n_atoms][25][n_rad], distinct arrays. */
int lasto_op_sphere_density(const lasto_cluster* cl, int n_rad, double r_min, int n_theta, int n_phi, double* rho_lm,
                            int* status, void* stream);
int lasto_op_inner_solve(int n_atoms, const double* R, const double* Z, int n_rad, double r_min, const double* rho_lm,
                         const double* v_R, double* v, void* stream);

/* Learned initial guess.  The paper has no counterpart: it solves every SCF step from
 * scratch.  A small 3-D U-Net (four levels, 16-32-64-64 channels, 3x3x3 convolutions with
 * BF16 tensor-core products and FP32 accumulation) maps the right-hand side restricted to a
 * 33^3 subgrid of the mesh (every m-th node, m = (n - 1) / 32), the subgrid's Dirichlet
 * faces and its local mesh size to the subgrid potential; carried up the multigrid
 * hierarchy by trilinear prolongation it is the first iterate.  The iteration then runs to
 * the same tolerance, so the network changes how many iterations a solve takes, never what
 * it converges to.
 * params: host FP32, the 15 convolutions in the order e1a e1b e2a e2b e3a e3b bta btb d3a d3b
 * d2a d2b d1a d1b out (cin->cout: 16-16, 16-16, 16-32, 32-32, 32-64, 64-64, 64-64, 64-64,
 * 128-64, 64-64, 96-32, 32-32, 48-16, 16-16, 16-16), each as weights [27][cin][cout]
 * (tap = (dz+1)*9 + (dy+1)*3 + (dx+1)) followed by its bias [cout];
 * n_params = lasto_guess_param_count().  scales = {s0, s1, h_ref, out}: input channel 0 is
 * b h^2 s0, channel 1 the face value s1, channel 2 log(h / h_ref); the potential is the
 * prediction / out.  Copied to the device (synchronously); later solves use the network for
 * every cluster whose axes all have 32 m + 1 nodes, when the caller passes no guess.
 * params == NULL removes the network.  INVALID_ARG for a wrong count or a zero scale. */
size_t lasto_guess_param_count(void);
int lasto_poisson_set_guess(lasto_poisson* h, const float* params, size_t n_params, const double scales[4]);

/* Allocates the workspace for cfg (device memory sized by n_max, max_atoms,
 * max_batch).  *out is NULL on failure.  Errors: INVALID_ARG, CUDA, NO_MEMORY. */
int lasto_poisson_create(const lasto_config* cfg, lasto_poisson** out);

/* The whole step (Section 3, Eq. 3.2-3.6) for n_clusters clusters (<= max_batch).
 *   v_lm      device [sum n_atoms][25]: V_LM(R_i) = int y_LM V dOmega on each sphere
 *             surface (Eq. 3.6; reading: unit-sphere measure so V = sum V_LM y_LM).
 *   potential device, optional (NULL): the converged u of every cluster,
 *             concatenated grids.
 *   guess     device, optional (NULL): interior initial guess, same layout as
 *             potential (faces are overwritten by the multipole values).
 *   stats     host [n_clusters], optional (NULL); written from the stream after the
 *             solve (valid after stream sync); must stay alive until then.
 * The handle replays a CUDA graph captured for the same pointers and sizes, so
 * repeated solves on the same buffers cost one graph launch; solves may be enqueued
 * back to back without synchronising, each filling its own stats.  New pointers or
 * sizes recapture the graph: that call first waits for the handle's previous solve
 * to finish.  Not thread-safe per handle.  Device outcomes per cluster go to
 * stats[c].status. */
int lasto_poisson_solve(lasto_poisson* h, const lasto_cluster* clusters, int n_clusters, double* v_lm,
                        double* potential, const double* guess, lasto_stats* stats, void* stream);

/* Frees the handle after waiting for its last solve (and that solve's stats copy). */
void lasto_poisson_destroy(lasto_poisson* h);

/* Kernel launches of the graph captured by the last lasto_poisson_solve on h:
 * *fixed = kernels that run once per solve (setup, deposit, multipoles, faces,
 * projection, ...), *per_iteration = kernels in one CG iteration or V-cycle,
 * *per_outer = kernels of one defect-correction step outside its inner iterations
 * (0 unless MIXED with CG); one solve launches
 * fixed + cycles * per_iteration + outer * per_outer kernels (stats.cycles,
 * stats.outer).  Host pointers.  Errors: INVALID_ARG if no graph was captured yet. */
int lasto_poisson_kernel_counts(const lasto_poisson* h, int* fixed, int* per_iteration, int* per_outer);

/* Text of the last error on this handle (never NULL; "" when none). */
const char* lasto_poisson_last_error(const lasto_poisson* h);

/* ------------------------------------------------------------------ mesh (Section 3)
 * One mesh axis, "fine meshes near the atoms and coarse meshes at large distances"
 * with Dirichlet conditions at the edge (Section 3, first paragraph):
 *   x(xi) = centre + A xi + B sign(xi)|xi|^p, xi = (i - m)/m, m = (n-1)/2,
 *   A = h_min m, A + B = half_width, A + p B = h_max m; when p > p_max, p = p_max
 *   and A, B follow from the other two conditions; B = 0 gives a uniform axis.
 * x: device [n].  info: device [5] = {A, B, p, centre spacing, edge spacing}, may be NULL.
 * Errors (host-checked): INVALID_ARG for even n, n < 3, or parameters with no
 * monotone solution. */
int lasto_mesh_axis(int n, double centre, double half_width, double h_min, double h_max, double p_max,
                    double* x, double* info, void* stream);

/* ------------------------------------------------------------------ single operations
 * Each runs one kernel family of the solve on caller buffers, for parity tests
 * and for callers composing their own pipeline.  They allocate their own small
 * scratch with the stream-ordered allocator and free it on the same stream. */

/* Per-sphere pseudo-density (Section 3, the three constraints beside Eq. 3.2-3.3;
 * reading: rho_tilde = a + b r^2 + c r^4).  Outputs device [n_atoms]: q (charge of
 * rho - Z delta inside the sphere, electron sign), rhoR, drhoR (monopole of the
 * density and its slope at R), coef [n_atoms][3] = (a, b, c).  status: device int,
 * set to GEOMETRY if spheres overlap, INVALID_ARG if zeta differs between atoms,
 * left unchanged otherwise (caller zeroes it). */
int lasto_op_sphere_params(const lasto_cluster* cl, double* q, double* rhoR, double* drhoR, double* coef,
                           int* status, void* stream);

/* Deposit b = 4 pi rho_tilde_grid at every node (Section 1's pseudo-density swap):
 * inside sphere i, n_e - rho0_i(r) + rho_tilde_i(r); elsewhere n_e.  owner: device
 * int [N] (sphere index or -1), may be NULL.  precision selects FP64 or FP32-pair
 * exponentials.  status as above, plus NONFINITE. */
int lasto_op_deposit(const lasto_cluster* cl, int precision, double* b, int* owner, int* status, void* stream);

/* Allocation-free variant of lasto_op_deposit, for callers that cannot allocate device
 * memory when they deposit (a fixed device-memory budget set at start-up, a device heap
 * owned by another framework's allocator, a real-time loop that forbids allocation).
 * The paper has no counterpart: this is a property of the library, not of the method.
 * Same arguments, kernels and results as lasto_op_deposit; the per-sphere records live
 * in one file-scope device array sized for 1024 atoms (384 KiB, held by every device
 * that loads the library until exit) instead of allocator scratch.  No cudaMalloc,
 * cudaFree or allocating library routine is called.
 * b (and owner, when given) must hold N = n0 n1 n2 elements: the entry point takes no
 * lengths and writes all N.  status may be NULL; when given, the caller zeroes it first
 * (the kernels only raise it, so a stale nonzero value would be carried into the result).
 * Errors: INVALID_ARG when n_atoms > 1024 (or as lasto_op_deposit, grid checks included),
 * CUDA when the array's device address cannot be found or a launch fails.
 * The first call on each device looks up that address (and uploads the constant tables)
 * with the device current; make that first call before any stream capture.  Every call
 * shares the one array: calls that overlap on the GPU (two streams, or two host threads)
 * race and must be ordered by the caller. */
int lasto_op_deposit_noalloc(const lasto_cluster* cl, int precision, double* b, int* owner, int* status,
                             void* stream);

/* Boundary multipoles Q_lm = sum_nodes (b/4pi) vol r^l y_lm(node - centre), l <= 4,
 * vol = product of dual-cell lengths.  Q: device [25]. */
int lasto_op_multipoles(const int n[3], const double* x, const double* y, const double* z, const double* b,
                        const double centre[3], double* Q, void* stream);

/* Dirichlet faces u = -sum_lm 4pi/(2l+1) Q_lm y_lm / r^(l+1) about centre (Eq. 2.7
 * decay).  Writes only the six faces of u. */
int lasto_op_boundary_fill(const int n[3], const double* x, const double* y, const double* z,
                           const double centre[3], const double* Q, double* u, void* stream);

/* The six faces of u set to the exact superposition of the atoms' continuum potentials
 * (LASTO_BC_EXACT); the cluster's arrays and axes are device arrays. */
int lasto_op_boundary_exact(const lasto_cluster* cl, double* u, void* stream);

/* Au = A u on interior nodes (7-point nonuniform difference), 0 on faces. */
int lasto_op_apply(const int n[3], const double* x, const double* y, const double* z, const double* u,
                   double* Au, void* stream);

/* r = b - A u on interior nodes, 0 on faces. */
int lasto_op_residual(const int n[3], const double* x, const double* y, const double* z, const double* u,
                      const double* b, double* r, void* stream);

/* Red-black Gauss-Seidel (Section 3): `sweeps` sweeps, each a red (i+j+k even) then a black
 * half sweep, in place on u (FP64, or FP32 for the _f32 form).  threads: 32..512 (a multiple
 * of 32) threads per block over the flat node index, or 0 for one block per (j, k) row (rows
 * of at most 1023 nodes); every choice gives bitwise the same result. */
int lasto_op_smooth(const int n[3], const double* x, const double* y, const double* z, double* u,
                    const double* b, int sweeps, int threads, void* stream);
int lasto_op_smooth_f32(const int n[3], const double* x, const double* y, const double* z, float* u,
                        const float* b, int sweeps, int threads, void* stream);

/* The same FP32 sweeps over colour-split storage, the layout the solver gives its finest FP32
 * level when the smoother tuner finds it faster: u and b hold the red nodes (even flat index
 * P = i + n0 (j + n1 k), i.e. i+j+k even, every axis odd) in flat order at P / 2, then the
 * black ones at (P - 1) / 2 + ceil(N / 2), N = n0 n1 n2.  Each half sweep then reads only the
 * other colour and its own right-hand side and writes only its own colour, all with unit
 * stride.  Bitwise the result of lasto_op_smooth_f32 on the same values in natural order.
 * threads: as lasto_op_smooth_f32 (0: one warp per row, rows of at most 513 nodes), or 1 for
 * the plane-staged kernel (a block marches a tile of 8 rows through a chunk of planes with the
 * other colour's planes bulk-copied into shared memory one plane ahead; every axis at least 9
 * nodes, rows of at most 513, u and b 16-byte aligned; this form synchronises the stream at the
 * end and returns LASTO_ERR_TIMEOUT if one of its bounded device waits ran out).
 * INVALID_ARG also for an even axis. */
int lasto_op_smooth_split_f32(const int n[3], const double* x, const double* y, const double* z, float* u,
                              const float* b, int sweeps, int threads, void* stream);

/* Red-black Gauss-Seidel on z-slabs staged in shared memory (the Section 3 smoother):
 * `sweeps` full sweeps, each colour `first` (0 = red, i+j+k even) then the other, from
 * u_in into u_out, fused ns (1 or 2) sweeps per pass over the grid.  u_in, u_out, b:
 * distinct device arrays [n0*n1*n2] (x fastest); u_in is not modified; every node of
 * u_out is written, faces copied from u_in.  The result is bitwise that of `sweeps`
 * in-place sweeps.  tile = {tx, ty, kz}: the (x, y) tile and the number of z planes one
 * thread block owns (any tile gives the same result).  ns = 1 passes need tx = 62 and
 * 32 (ty + 2) threads <= 512 (FP32) or 256 (FP64); ns = 2 passes take any tile within the
 * shared-memory limit; a remainder pass (sweeps not a multiple of ns) runs the one-sweep
 * kernel on its own tile with the given kz.  More than one pass takes one
 * device scratch grid from the stream-ordered allocator.  INVALID_ARG for sweeps < 1, ns
 * outside {1, 2}, a tile needing more than 200 KiB of shared memory, or u_in == u_out. */
int lasto_op_smooth_slab(const int n[3], const double* x, const double* y, const double* z, const double* u_in,
                         double* u_out, const double* b, int sweeps, int ns, int first, const int tile[3],
                         void* stream);
int lasto_op_smooth_slab_f32(const int n[3], const double* x, const double* y, const double* z, const float* u_in,
                             float* u_out, const float* b, int sweeps, int ns, int first, const int tile[3],
                             void* stream);

/* Red-black Gauss-Seidel (Section 3) as fused FP32 passes, one full sweep per pass, each
 * walking z as a wavefront over row chunks staged in shared memory: the first colour of
 * plane k+1, then the other colour of plane k.  `sweeps` sweeps, each colour `first` (0 =
 * red, i+j+k even) then the other, from u_in into u_out (distinct, 16-byte aligned device
 * arrays [n0*n1*n2], x fastest; u_in unchanged; every node of u_out written, faces copied).
 * Bitwise the result of `sweeps` in-place sweeps.  tx (16..60) columns and ty (8, 12 or 16)
 * rows per thread-block tile (any tile gives the same result); rows of at least 69 nodes.
 * More than one sweep takes one device scratch grid from the stream-ordered allocator.
 * INVALID_ARG for sweeps < 1, a bad tile, a short row, misaligned arrays or u_in == u_out. */
int lasto_op_smooth_wave_f32(const int n[3], const double* x, const double* y, const double* z, const float* u_in,
                             float* u_out, const float* b, int sweeps, int first, int tx, int ty, void* stream);

/* Self-test of the bounded device waits (the paper has no counterpart).  The staged
 * tensor-core kernels (the H/S contraction, the convolution of the learned guess) wait on
 * mbarriers with a time limit and, when it runs out, raise
 * LASTO_ERR_TIMEOUT in a device status and return instead of hanging.  This entry launches
 * one thread that waits on an mbarrier nothing ever arrives at, for `seconds` (0 < s <= 60),
 * and then raises *status (device int, caller-zeroed) to LASTO_ERR_TIMEOUT the same way.
 * Asynchronous on the stream; the stream stays usable afterwards. */
int lasto_selftest_bounded_wait(double seconds, int* status, void* stream);

/* Arithmetic throughput probe (the paper has no counterpart): `blocks` blocks of 256
 * threads, each thread 8 independent fused multiply-add chains of 16 * iters steps, in FP64
 * (precision 0) or FP32 (precision 1); out: device array of blocks * 256 elements of that
 * type (written, so nothing is folded away).  Work: 2 * 8 * 16 * iters FLOP per thread.  It
 * measures the ALU ceilings the roofline of the ALU-bound kernels is stated against. */
int lasto_probe_fma(int precision, int blocks, int iters, void* out, void* stream);

/* Full weighting bc = Vc^-1 P^T Vf r onto the every-other-node mesh; bc device
 * [(n0+1)/2 * (n1+1)/2 * (n2+1)/2], faces set to 0.  x, y, z are the fine axes. */
int lasto_op_restrict(const int n[3], const double* x, const double* y, const double* z, const double* r,
                      double* bc, void* stream);

/* u += P ec on fine interior nodes, P = trilinear interpolation in physical
 * coordinates; ec is the coarse field (faces are read as stored). */
int lasto_op_prolong_add(const int n[3], const double* x, const double* y, const double* z, const double* ec,
                         double* u, void* stream);

/* Exact solve A e = b on a grid of at most 9 nodes per axis with zero faces (fast
 * diagonalisation of the three 1-D operators).  e faces set to 0. */
int lasto_op_coarse_solve(const int n[3], const double* x, const double* y, const double* z, const double* b,
                          double* e, void* stream);

/* V_LM(R_i) of Eq. 3.6 for n_atoms spheres: n_theta Gauss-Legendre points in
 * cos(theta) x n_phi uniform phi; trilinear interpolation of u in physical
 * coordinates.  vlm device [n_atoms][25].  status: GEOMETRY if a surface point
 * leaves the box. */
int lasto_op_project(const int n[3], const double* x, const double* y, const double* z, const double* u,
                     int n_atoms, const double* pos, const double* R, int n_theta, int n_phi, double* vlm,
                     int* status, void* stream);

/* ------------------------------------------------------------------ learned initial guess
 * Operations of the small 3-D U-Net that predicts the coarse-grid (33^3) potential used as the
 * multigrid initial guess.  The paper has no counterpart (it solves from scratch each SCF
 * step); the network is an accelerator: multigrid always runs to the same residual, so the
 * guess changes only the iteration count, never the answer.
 * Layout: channels-last, [node][channel], node = ((b*D + z)*H + y)*W + x over nb grids of
 * dims = {W, H, D} nodes.  Weights: [27 taps][cin][cout], tap = (dz+1)*9 + (dy+1)*3 + (dx+1),
 * zero padding.  BF16 arrays are passed as void* (2 bytes per element); cin, cout multiples
 * of 16 (cout <= 128; wgrad cout <= 64).  All pointers device; all calls asynchronous;
 * INVALID_ARG for unsupported sizes, CUDA for launch failures. */

/* y = act(conv(x, w) + bias), act = ReLU if relu != 0.  Tensor-core BF16 products, FP32
 * accumulation.  y32 (FP32, row stride ldy32, channel offset off32) and y16 (BF16, ldy16,
 * off16) are each optional: writing into a channel slice makes concatenation free. */
int lasto_nn_conv3d_fwd(int nb, const int dims[3], int cin, int cout, const void* x, const void* w, const float* bias,
                        int relu, float* y32, int ldy32, int off32, void* y16, int ldy16, int off16, void* stream);
/* The forward convolution on the fifth-generation tensor cores (tcgen05.mma, accumulator in
 * tensor memory), same arguments and results as lasto_nn_conv3d_fwd except the weights,
 * which are packed once by lasto_nn_pack_weights (same size, 27*cin*cout BF16) into the
 * per-step operand tiles.  cout in {16, 32, 48, 64, 96, 128}.  err (device int, optional) is
 * set to 1 if a tensor-core completion wait timed out (the outputs are then not written). */
int lasto_nn_pack_weights(int cin, int cout, const void* w, void* wpk, void* stream);
int lasto_nn_conv3d_fwd_tc(int nb, const int dims[3], int cin, int cout, const void* x, const void* wpk,
                           const float* bias, int relu, float* y32, int ldy32, int off32, void* y16, int ldy16,
                           int off16, int* err, void* stream);
/* dx32 = data gradient of the convolution for output gradient dy (BF16 [node][cout]);
 * w_flip is caller scratch of 27*cin*cout BF16 (the flipped, transposed weights). */
int lasto_nn_conv3d_dgrad(int nb, const int dims[3], int cin, int cout, const void* dy, const void* w, void* w_flip,
                          float* dx32, void* stream);
/* dw (FP32 [27][cin][cout]) += weight gradient; db (FP32 [cout], optional) += bias gradient
 * from dy32 (FP32 copy of dy).  dw accumulates with atomics (order not fixed). */
int lasto_nn_conv3d_wgrad(int nb, const int dims[3], int cin, int cout, const void* x, const void* dy16,
                          const float* dy32, float* dw, float* db, void* stream);
/* The data and weight gradients on the fifth-generation tensor cores (the paper has no
 * counterpart; training of the learned guess).  dgrad_tc: as lasto_nn_conv3d_dgrad, the
 * flipped weights packed into wpk_flip (caller scratch, 27*cin*cout BF16) and convolved with
 * dy by the tcgen05 forward kernel; cin in {16, 32, 48, 64, 96, 128}.  wgrad_tc: as
 * lasto_nn_conv3d_wgrad, as a tcgen05 GEMM over the nodes (M = rows of (tap, input channel),
 * N = cout, both operands read from the channels-last rows), cin <= 128, cout in {16, 32,
 * 48, 64, 96, 128}.  err (device int, optional) is set to 1 if a tensor-core completion wait
 * timed out (dx32 / dw are then incomplete). */
int lasto_nn_conv3d_dgrad_tc(int nb, const int dims[3], int cin, int cout, const void* dy, const void* w, void* w_flip,
                             void* wpk_flip, float* dx32, int* err, void* stream);
int lasto_nn_conv3d_wgrad_tc(int nb, const int dims[3], int cin, int cout, const void* x, const void* dy16,
                             const float* dy32, float* dw, float* db, int* err, void* stream);
/* dx = dy where y > 0 else 0 (FP32 and / or BF16 output). */
int lasto_nn_relu_grad(size_t n, const float* y, const float* dy, float* dx, void* dx16, void* stream);
int lasto_nn_to_bf16(size_t n, const float* a, void* b, void* stream);
/* dst[node][doff + c] = (or +=) src[node][soff + c], c < C. */
int lasto_nn_copy_channels(size_t nodes, int C, const float* src, int lds, int soff, float* dst, int ldd, int doff,
                           int accumulate, void* stream);
/* Full-weighting average from a fine node grid (odd dims) onto every other node, boundary
 * planes renormalised; adjoint != 0 applies the transpose (coarse -> fine). */
int lasto_nn_down(int nb, const int fine[3], int C, const float* x, float* y, int adjoint, void* stream);
/* Trilinear interpolation from the every-other-node grid onto the fine grid, written into
 * channels [off, off + C) of rows of stride ldy; adjoint != 0: fine (ldy, off) -> coarse. */
int lasto_nn_up(int nb, const int fine[3], int C, const float* x, float* y, int ldy, int off, int adjoint, void* stream);
/* Masked mean-square error: loss (FP64, accumulated) += sum mask (p - t)^2 * inv_count and
 * dp = 2 mask (p - t) inv_count.  mask may be NULL. */
int lasto_nn_mse(size_t n, const float* p, const float* t, const float* mask, float inv_count, float* dp, double* loss,
                 void* stream);
/* Network input on the coarse (33^3) grid n[3] with coordinates x, y, z: out [N][16] FP32,
 * channel 0 = b h^2 s0 (interior), channel 1 = faces s1 (faces only), channel 2 = log(h/h_ref),
 * h the local dual-cell size; b and faces FP64 grids (faces: Dirichlet values, any interior). */
int lasto_nn_guess_features(const int n[3], const double* b, const double* faces, const double* x, const double* y,
                            const double* z, float s0, float s1, float h_ref, float* out, void* stream);
/* Coarse-grid guess u (FP64) = pred[node * ld] / scale inside, faces copied from `faces`. */
int lasto_nn_guess_grid(const int n[3], const float* pred, int ld, float scale, const double* faces, double* u,
                        void* stream);
/* One Adam step (Kingma & Ba) on FP32 master weights, step counted from 1; w16 (BF16 copy)
 * optional. */
int lasto_nn_adam(size_t n, float* w, const float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                  int step, void* w16, void* stream);

/* Interstitial overlap and Hamiltonian contributions (Section 3, Eq. 3.11-3.14, the
 * grid-point form of the interstitial integrals) of a Slater-type basis: over the nodes
 * outside every sphere (|P - pos_a| < R_a excludes a node), with Vol(P) the dual-cell volume,
 *   S_ab = sum_P phi_a phi_b Vol,  H_ab = 1/2 sum_P (phi_a phi~_b + phi~_a phi_b) Vol,
 * phi = r^(n-1) e^{-zeta r} y_lm about the function's atom (Eq. 3.13) and
 * phi~ = -1/2 Lap phi + V phi (Eq. 3.14, the radial Laplacian in closed form).
 * Basis (HOST arrays of nb <= 8 entries): principal number bn >= bl + 1, angular number
 * bl <= 4, exponent bz > 0; per atom sum(2 bl + 1) <= 64 functions.  Functions are
 * atom-major, then in the table's order, then m = -l..l (y_lm the real harmonics of the
 * solver's projections).  Device arrays: x, y, z node coordinates [n[d]]; pos [n_atoms][3];
 * R [n_atoms]; V the potential energy at the nodes [n[2]][n[1]][n[0]] (x fastest);
 * S, H [M][M] with M = n_atoms * functions per atom, written whole (symmetric).
 * Basis values in FP32 (weighted by sqrt(Vol)); mode LASTO_HS_TENSOR (the default) contracts
 * them on the tensor cores: each value, scaled by a power of two per function (one more
 * common power of two for phi~) below 2^14, is split into two FP16 parts and a product taken
 * as hi*hi + hi*lo + lo*hi (22 significant bits), FP32 accumulation over 512-node intervals
 * added in FP64 with the scales undone; LASTO_HS_SIMT takes FP32 products summed over 32-node
 * steps, added in FP64.  Sums across CTAs meet by FP64 atomic addition, so the last bits may
 * differ between calls.  Allocates its scratch stream-ordered (at most about 2 GiB of basis
 * tables, 8 bytes per node and 256 KiB per SM) and synchronises the stream twice.  INVALID_ARG for bad sizes, basis or mode,
 * n[0] n[1] n[2] >= 2^31 or M > 65536; NO_MEMORY when the scratch cannot be had; TIMEOUT when
 * a bounded wait of the tensor-core kernel ran out (outputs then undefined). */
enum lasto_hs_mode { LASTO_HS_DEFAULT = 0, LASTO_HS_SIMT = 1, LASTO_HS_TENSOR = 2 };
/* stats (host, may be NULL): what the call did and the device time of its stages (CUDA events
 * on the stream; all chunks summed). */
typedef struct lasto_hs_stats {
    long long interstitial_nodes;   /* nodes outside every sphere */
    int chunks;                     /* basis-table chunks */
    int tile;                       /* tile side of the contraction: 128 tensor, 64 SIMT */
    float ms_list;                  /* interstitial node list */
    float ms_tables;                /* basis tables */
    float ms_contract;              /* contraction */
    float ms_mirror;                /* lower triangle and the 1/2 of H */
} lasto_hs_stats;
int lasto_op_interstitial_hs(const int n[3], const double* x, const double* y, const double* z, int n_atoms,
                             const double* pos, const double* R, int nb, const int* bn, const int* bl, const double* bz,
                             const double* V, double* S, double* H, int mode, lasto_hs_stats* stats, void* stream);

#ifdef __cplusplus
}
#endif
#endif
