// Sphere-surface projection V_LM(R_i) = int y_LM V dOmega (Eq. 3.6), with V from
// trilinear interpolation of the grid potential ("interpolates onto the sphere
// boundaries", Section 1).  Reading of the measure: the unit-sphere solid angle, so
// that V = sum_LM V_LM y_LM on the surface (Eq. 3.5).  The quadrature is
// Gauss-Legendre in cos(theta) times uniform phi; the unit vectors and the weighted
// harmonics w_q y_LM(u_q) are mesh independent and built once on the host.
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace lasto {

// Gauss-Legendre nodes on [-1, 1]: Newton's method on P_n from the asymptotic guess
// cos(pi (i - 1/4) / (n + 1/2)), P_n and P_n' from the three-term recurrence.
static void gauss_legendre(int n, std::vector<double>& t, std::vector<double>& w)
{
    t.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 1; i <= n; i++) {
        double x = std::cos(PI * (i - 0.25) / (n + 0.5));
        double dpn = 1.0;
        for (int it = 0; it < 60; it++) {
            double pm = 1.0, pc = x;
            for (int k = 1; k < n; k++) {
                const double pn = ((2 * k + 1) * x * pc - k * pm) / (k + 1);
                pm = pc;
                pc = pn;
            }
            if (n == 1) pm = 1.0;
            dpn = n * (pm - x * pc) / (1.0 - x * x);
            const double dx = pc / dpn;
            x -= dx;
            if (std::fabs(dx) < 1e-17) break;
        }
        t[n - i] = x;
        w[n - i] = 2.0 / ((1.0 - x * x) * dpn * dpn);
    }
}

void host_quadrature(int n_theta, int n_phi, double* table)
{
    std::vector<double> ct, wt;
    gauss_legendre(n_theta, ct, wt);
    int q = 0;
    for (int a = 0; a < n_theta; a++) {
        const double st = std::sqrt(std::max(0.0, 1.0 - ct[a] * ct[a]));
        for (int b = 0; b < n_phi; b++, q++) {
            const double ph = 2.0 * PI * b / n_phi;
            const double ux = st * std::cos(ph), uy = st * std::sin(ph), uz = ct[a];
            double S[NLM];
            host_solid_harmonics(ux, uy, uz, S);
            double* row = table + (size_t)q * 28;
            row[0] = ux;
            row[1] = uy;
            row[2] = uz;
            const double wq = wt[a] * 2.0 * PI / n_phi;
            for (int lm = 0; lm < NLM; lm++) row[3 + lm] = wq * S[lm];
        }
    }
}

// largest i with c[i] <= p, clamped to [0, n-2]
__device__ __forceinline__ int cell_of(const double* __restrict__ c, int n, double p)
{
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (c[mid] <= p) lo = mid;
        else hi = mid;
    }
    if (c[hi] <= p) lo = hi;
    return lo > n - 2 ? n - 2 : lo;
}

constexpr int PRJ_NT = 256;

__global__ void __launch_bounds__(PRJ_NT) k_project(int nx, int ny, int nz, const double* __restrict__ x,
                                                   const double* __restrict__ y, const double* __restrict__ z,
                                                   const double* __restrict__ u, const double* __restrict__ pos,
                                                   const double* __restrict__ R, const double* __restrict__ quad,
                                                   int nq, double* __restrict__ vlm, int* status)
{
    __shared__ double sm[32];
    const int a = blockIdx.x;
    const double cx = pos[3 * a], cy = pos[3 * a + 1], cz = pos[3 * a + 2], Ra = R[a];
    double acc[NLM];
#pragma unroll
    for (int lm = 0; lm < NLM; lm++) acc[lm] = 0.0;
    int bad = 0;
    for (int q = threadIdx.x; q < nq; q += PRJ_NT) {
        const double* row = quad + (size_t)q * 28;
        const double px = fma(Ra, row[0], cx), py = fma(Ra, row[1], cy), pz = fma(Ra, row[2], cz);
        if (!(px >= x[0] && px <= x[nx - 1] && py >= y[0] && py <= y[ny - 1] && pz >= z[0] && pz <= z[nz - 1])) {
            bad = 1;
            continue;
        }
        const int i = cell_of(x, nx, px), j = cell_of(y, ny, py), k = cell_of(z, nz, pz);
        const double tx = (px - x[i]) / (x[i + 1] - x[i]);
        const double ty = (py - y[j]) / (y[j + 1] - y[j]);
        const double tz = (pz - z[k]) / (z[k + 1] - z[k]);
        const size_t sy = nx, sz = (size_t)nx * ny;
        const double* c0 = u + (size_t)k * sz + (size_t)j * sy + i;
        const double v00 = fma(tx, c0[1] - c0[0], c0[0]);
        const double v10 = fma(tx, c0[sy + 1] - c0[sy], c0[sy]);
        const double v01 = fma(tx, c0[sz + 1] - c0[sz], c0[sz]);
        const double v11 = fma(tx, c0[sz + sy + 1] - c0[sz + sy], c0[sz + sy]);
        const double v0 = fma(ty, v10 - v00, v00), v1 = fma(ty, v11 - v01, v01);
        const double V = fma(tz, v1 - v0, v0);
#pragma unroll
        for (int lm = 0; lm < NLM; lm++) acc[lm] = fma(V, row[3 + lm], acc[lm]);
    }
    for (int lm = 0; lm < NLM; lm++) {
        const double s = block_sum<PRJ_NT>(acc[lm], sm);
        if (threadIdx.x == 0) vlm[(size_t)NLM * a + lm] = s;
    }
    if (bad && status) atomicMax(status, (int)LASTO_ERR_GEOMETRY);
}

cudaError_t launch_project(const int n[3], const double* x, const double* y, const double* z, const double* u,
                           int n_atoms, const double* pos, const double* R, const double* quad, int nq,
                           double* vlm, int* status, cudaStream_t s)
{
    if (n_atoms <= 0) return cudaSuccess;
    k_project<<<n_atoms, PRJ_NT, 0, s>>>(n[0], n[1], n[2], x, y, z, u, pos, R, quad, nq, vlm, status);
    return cudaGetLastError();
}

}  // namespace lasto
